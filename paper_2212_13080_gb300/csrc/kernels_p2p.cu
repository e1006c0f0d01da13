// Evaluation at the charges: near field (step 5: direct sum over the finest
// cell and its 26 neighbours) and far field (§2.2 step 4 and the far-field force
// at the end of §2.2).  Results in unit-box units, (phi, F_x, F_y, F_z) with phi
// per unit charge and F with the charge.
// The near-field kernel evaluates every pair of neighbouring cells once for
// both partners (mutual form): it writes the target cell's own sums to
// out_pt[slot] (sorted order) and the partners' reactions to one slot per
// direction; the far-field kernel adds the slots in a fixed order and the far
// field, and stores the total by emitted index, out_e[perm[slot]], where the
// recombination reads each particle's charges in a row.  The near field needs
// only the sorted charges and runs beside the far field.
#include "fmm_internal.cuh"
#include "lagrange.cuh"
#include "launch.cuh"

#ifndef NF_QUNROLL
#define NF_QUNROLL 16  // unroll of the target-pair loop of the packed evaluation
#endif

namespace fmm {

__device__ __forceinline__ float4 make_vec4(float a, float b, float c, float d) { return make_float4(a, b, c, d); }
__device__ __forceinline__ double4 make_vec4(double a, double b, double c, double d) {
    return make_double4(a, b, c, d);
}

// Near-field directions: index 13 + d of the 3x3x3 block (x fastest) for
// d = 0..13, i.e. the cell itself (d = 0) and the 13 neighbours that come
// after it in (z, y, x) order.  Every unordered pair of neighbouring cells
// {A, A + delta_d} is evaluated once, by the CTA of A.
#define NF_SEGS 14
__host__ __device__ __forceinline__ void nf_delta(int d, int &dx, int &dy, int &dz) {
    const int i = 13 + d;
    dx = i % 3 - 1;
    dy = (i / 3) % 3 - 1;
    dz = i / 9 - 1;
}
// Cell reached from (cx, cy, cz) by (dx, dy, dz), wrapped (periodic) or -1
// outside the box (open).
__device__ __forceinline__ int64_t nf_cell(int cx, int cy, int cz, int dx, int dy, int dz, int S,
                                           int periodic) {
    int nx = cx + dx, ny = cy + dy, nz = cz + dz;
    if (periodic) {
        nx = (nx + S) % S;
        ny = (ny + S) % S;
        nz = (nz + S) % S;
    } else if (nx < 0 || ny < 0 || nz < 0 || nx >= S || ny >= S || nz >= S) {
        return -1;
    }
    return (int64_t)morton_encode(nx, ny, nz);
}

// ---------------------------------------------------------------------------
// far field: phi_far = sum_ijk g_i(t_x) g_j(t_y) g_k(t_z) L_leaf[ijk] and
// F_far = -q * 2^depth * grad_t phi_far.  KF (force kernels, §4.1): the far
// force is q times the plain weights against the three force functionals,
// F_far,c = q g(t) . L^c_leaf.  One CTA per four consecutive finest cells
// (their charges are one contiguous range; one cell when the four cells'
// functionals would not fit the static shared memory), L_leaf in shared
// memory, one thread per charge.
// ---------------------------------------------------------------------------
#define L2P_BS 128
#ifndef L2P_LPC
#define L2P_LPC 4  // finest cells per CTA (consecutive keys: one contiguous charge range)
#endif

template <typename real, int P, bool KF>
constexpr int l2p_lpc() {
    return (KF && (size_t)L2P_LPC * 4 * P * P * P * sizeof(real) > 24576) ? 1 : L2P_LPC;
}

template <typename real, int P, bool FORCES, bool KF>
struct KL2P {
    static constexpr int BS = L2P_BS, MINB = 0;  // bounds on the block size only
    Coef<real> C;
    int depth;
    int periodic;
    int ncell;
    int sf;
    const int *__restrict__ leaf_start;
    const typename Vec4<real>::T *__restrict__ s_pt;
    const real *__restrict__ loc_leaf;
    int64_t loc_comp;
    const typename Vec4<real>::T *__restrict__ react;
    int64_t rstride;
    const typename Vec4<real>::T *__restrict__ out_pt;
    const int *__restrict__ perm;
    typename Vec4<real>::T *__restrict__ out_e;
    __device__ __forceinline__ void run(const int bid_, const int nblk_) const {
        typedef typename Vec4<real>::T real4;
        constexpr int P3 = P * P * P;
        constexpr int LPC = l2p_lpc<real, P, KF>();
        constexpr int NCL = KF ? 4 : 1;  // functionals per cell: potential (+ 3 force components)
        __shared__ real Ls[LPC][NCL][P3];
        __shared__ int slot_ok[LPC][NF_SEGS - 1];
        __shared__ int lst[LPC + 1];
        __shared__ real org[LPC][3];  // coordinate of the weights: org + h t
        const int k0 = bid_ * LPC;
        const int nleaf = min(LPC, ncell - k0);
        if (threadIdx.x <= LPC) lst[threadIdx.x] = leaf_start[min(k0 + (int)threadIdx.x, ncell)];
        __syncthreads();
        if (lst[0] == lst[nleaf]) return;  // no charges in these cells (the whole CTA)
        for (int e = threadIdx.x; e < nleaf * NCL * P3; e += blockDim.x) {
            const int j = e / (NCL * P3), c = (e / P3) % NCL, o = e % P3;
            if (lst[j + 1] == lst[j]) continue;  // an empty cell: its functionals are not read
            int cx, cy, cz;
            morton_decode((uint32_t)(k0 + j), cx, cy, cz);
            Ls[j][c][o] = loc_leaf[c * loc_comp + loc_cell(depth, cx, cy, cz) * P3 + o];
            if (c == 0 && o < 3) org[j][o] = sf ? (real)(o == 0 ? cx : o == 1 ? cy : cz) / (real)(1 << depth) : real(0);
        }
        // slot d - 1 of a cell's charges was written by the cell (that cell -
        // delta_d), d = 1..13, if it exists and holds charges
        if (threadIdx.x < nleaf * (NF_SEGS - 1)) {
            const int j = threadIdx.x / (NF_SEGS - 1), d = threadIdx.x % (NF_SEGS - 1);
            int cx, cy, cz, dx, dy, dz;
            morton_decode((uint32_t)(k0 + j), cx, cy, cz);
            nf_delta(d + 1, dx, dy, dz);
            const int64_t a = nf_cell(cx, cy, cz, -dx, -dy, -dz, 1 << depth, periodic);
            slot_ok[j][d] = a >= 0 && leaf_start[a + 1] > leaf_start[a];
        }
        __syncthreads();
        const real S = (real)(1 << depth);
        // cell-local weights (t) or, shift-free, box weights at (c + t)/2^depth;
        // the force is -q times the gradient in unit-box coordinates
        const real h = sf ? real(1) / S : real(1), FS = sf ? real(1) : S;
        for (int s = lst[0] + threadIdx.x; s < lst[nleaf]; s += blockDim.x) {
            int lf = 0;  // which of the CTA's cells holds charge s
            while (s >= lst[lf + 1]) lf++;
            const int *okc = slot_ok[lf];
            typename Vec4<real>::T v = s_pt[s];
            const real X = org[lf][0] + h * v.x, Y = org[lf][1] + h * v.y, Z = org[lf][2] + h * v.z;
            real gx[FMM_MAXP], gy[FMM_MAXP], gz[FMM_MAXP], dx[FMM_MAXP], dy[FMM_MAXP], dz[FMM_MAXP];
            if (FORCES && !KF) {
                lag_weights_deriv(C, P, X, gx, dx);
                lag_weights_deriv(C, P, Y, gy, dy);
                lag_weights_deriv(C, P, Z, gz, dz);
            } else {
                lag_weights(C, P, X, gx);
                lag_weights(C, P, Y, gy);
                lag_weights(C, P, Z, gz);
            }
            real phi = 0, fx = 0, fy = 0, fz = 0;
            if (KF) {
                const real *L0 = Ls[lf][0], *L1 = Ls[lf][NCL > 1 ? 1 : 0], *L2 = Ls[lf][NCL > 2 ? 2 : 0],
                           *L3 = Ls[lf][NCL > 3 ? 3 : 0];
#pragma unroll 1
                for (int k = 0; k < P; k++) {
                    real a0 = 0, a1 = 0, a2 = 0, a3 = 0;
#pragma unroll
                    for (int j = 0; j < P; j++) {
                        real r0 = 0, r1 = 0, r2 = 0, r3 = 0;
#pragma unroll
                        for (int i = 0; i < P; i++) {
                            const int o = (k * P + j) * P + i;
                            r0 += gx[i] * L0[o];
                            r1 += gx[i] * L1[o];
                            r2 += gx[i] * L2[o];
                            r3 += gx[i] * L3[o];
                        }
                        a0 += gy[j] * r0;
                        a1 += gy[j] * r1;
                        a2 += gy[j] * r2;
                        a3 += gy[j] * r3;
                    }
                    phi += gz[k] * a0;
                    fx += gz[k] * a1;
                    fy += gz[k] * a2;
                    fz += gz[k] * a3;
                }
            } else {
                const real *Lc = Ls[lf][0];
#pragma unroll 1
                for (int k = 0; k < P; k++) {
                    real ax = 0, ay = 0, az = 0, aw = 0;
#pragma unroll
                    for (int j = 0; j < P; j++) {
                        real rx = 0, rdx = 0;
#pragma unroll
                        for (int i = 0; i < P; i++) {
                            real Lv = Lc[(k * P + j) * P + i];
                            rx += gx[i] * Lv;
                            if (FORCES) rdx += dx[i] * Lv;
                        }
                        ax += gy[j] * rx;
                        if (FORCES) {
                            ay += gy[j] * rdx;
                            az += dy[j] * rx;
                            aw += gy[j] * rx;
                        }
                    }
                    phi += gz[k] * ax;
                    if (FORCES) {
                        fx += gz[k] * ay;
                        fy += gz[k] * az;
                        fz += dz[k] * aw;
                    }
                }
            }
            // near field: own sums, then the reactions of the 13 slots in order
            real4 o = out_pt[s];
#pragma unroll
            for (int d = 0; d < NF_SEGS - 1; d++) {
                if (!okc[d]) continue;
                const real4 r = react[d * rstride + s];
                o.x += r.x;
                o.y += r.y;
                o.z += r.z;
                o.w += r.w;
            }
            o.x += phi;
            if (KF) {  // the force functionals are in unit-box units already
                o.y += v.w * fx;
                o.z += v.w * fy;
                o.w += v.w * fz;
            } else {
                o.y += -v.w * FS * fx;
                o.z += -v.w * FS * fy;
                o.w += -v.w * FS * fz;
            }
            out_e[perm[s]] = o;
        }
    }
};
template <typename real, int P, bool FORCES, bool KF>
__global__ void __launch_bounds__(KL2P<real, P, FORCES, KF>::BS) k_l2p(const __grid_constant__ KL2P<real, P, FORCES, KF> k) {
    k.run(blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------------
// near field, mutual form.  One CTA of 128 threads per cell A.
//
// Forward phase: the source list is the charges of the 13 forward neighbours
// A + delta_d (d = 1..13), shifted into A's frame (source t + delta_d).  Each
// thread holds NF_KS sources in registers, with their reaction sums; A's
// charges (targets) are read from shared memory by all threads at once.  Every
// (target, source) pair is evaluated once and feeds both the target's sum
// (per group of targets: transposed through shared memory and summed over the
// warp's lanes in order, then over the four warps in order) and the source's
// reaction.  Charges of different cells coincide only in the continuous form
// with odd p, whose middle split charges sit on the cell plane (local
// coordinate 1 below it, 0 above); otherwise the frame coordinates differ by
// at least one ulp along an axis of delta_d.  So the pairs to skip are charges
// of the same particle (split charges) and, with odd p, coincident charges:
// CK = 0 (plain form: every charge is a particle of its own, none to skip),
// 1 (continuous form: charges of the same particle), 2 (and coincident ones).
// Single precision evaluates two targets per packed FP32x2 instruction
// (nf_targets2), the targets staged a second time by pairs.  A pass with at
// most 128 (256) sources evaluates the first one (two) of each thread's
// source slots only: slot k of thread t is source 128 k + t, so the count is
// the same for the whole CTA.  (Skipping empty slots warp by warp, with the
// slots assigned warp-major, was measured slower.)
//
// Own phase: the pairs inside A, one-sided (each target against all of A's
// charges), skipping charges of the same particle and coincident charges.
//
// Outputs: out_pt[A's charges] = A's own sums (assigned); react[d-1][j] = the
// reaction on charge j of A + delta_d, written by this CTA alone; the far-field
// kernel adds the 13 slots in order.  Large cells: sources in passes of
// 128 * NF_KS (the target sums accumulate in out_pt between passes), targets in
// blocks of TB (256 in single precision, 64 in double: static shared memory).
// ---------------------------------------------------------------------------
#define NF_BS 128
#define NF_KS 4  // source slots per thread
#ifndef NF_MINB
#define NF_MINB 4  // single precision: CTAs per SM the register allocation must allow
#endif
#define NF_TP 36  // row stride (words) of the per-warp transpose buffer

// Launch order of the near field: the occupied cells, heaviest first.  A
// cell's work grows with its charge count T (T times its own and its 13
// forward neighbours' charges), so the cells go in seven classes by T, the
// largest first, and within a class in the order the atomics hand out (a
// cell's sums do not depend on when its CTA runs: the results are the same
// bit for bit).  Clustered inputs put a few hundred cells with up to ~1000
// charges each among many light ones; launched in cell order they would
// start late and run alone at the end.  pord[0..6]: class sizes; pord[8..14]:
// fill counters; pord[16..]: the cells (zeroed before the count).
#define NF_NCLS 7
__device__ __forceinline__ int nf_class(int T) {
    return T >= 512 ? 0 : T >= 256 ? 1 : T >= 128 ? 2 : T >= 64 ? 3 : T >= 32 ? 4 : T >= 16 ? 5 : T > 0 ? 6 : -1;
}

struct KNfOrderCount {
    static constexpr int BS = 0, MINB = 0;
    int64_t ncell;
    const int *__restrict__ leaf_start;
    int *__restrict__ pord;
    __device__ __forceinline__ void run(const int bid_, const int nblk_) const {
        const int64_t c = bid_ * (int64_t)blockDim.x + threadIdx.x;
        const int cls = c < ncell ? nf_class(leaf_start[c + 1] - leaf_start[c]) : -1;
        const int lane = threadIdx.x & 31;
#pragma unroll
        for (int k = 0; k < NF_NCLS; k++) {
            const unsigned b = __ballot_sync(0xffffffffu, cls == k);
            if (lane == 0 && b) atomicAdd(&pord[k], __popc(b));
        }
    }
};
__global__ void k_nf_order_count(const __grid_constant__ KNfOrderCount k) {
    k.run(blockIdx.x, gridDim.x);
}

struct KNfOrderFill {
    static constexpr int BS = 0, MINB = 0;
    int64_t ncell;
    const int *__restrict__ leaf_start;
    int *__restrict__ pord;
    __device__ __forceinline__ void run(const int bid_, const int nblk_) const {
        const int64_t c = bid_ * (int64_t)blockDim.x + threadIdx.x;
        const int cls = c < ncell ? nf_class(leaf_start[c + 1] - leaf_start[c]) : -1;
        const int lane = threadIdx.x & 31;
        int first = 0;  // the first slot of class k
#pragma unroll
        for (int k = 0; k < NF_NCLS; k++) {
            const unsigned b = __ballot_sync(0xffffffffu, cls == k);
            int base = 0;
            if (lane == 0 && b) base = atomicAdd(&pord[8 + k], __popc(b));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (cls == k) pord[16 + first + base + __popc(b & ((1u << lane) - 1u))] = (int)c;
            first += pord[k];
        }
    }
};
__global__ void k_nf_order_fill(const __grid_constant__ KNfOrderFill k) {
    k.run(blockIdx.x, gridDim.x);
}

// 1/sqrt(r2): single precision uses the SFU reciprocal square root directly
// (r2 is never subnormal here: it is 0 or a squared distance of FP32 charges
// inside a few cells); double precision the correctly rounded form.
template <typename real> __device__ __forceinline__ real rsqrt_pair(real x);
template <> __device__ __forceinline__ float rsqrt_pair<float>(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
template <> __device__ __forceinline__ double rsqrt_pair<double>(double x) { return 1.0 / sqrt(x); }

// One (target, source) pair of the forward phase: target sums (p, x, y, z) in
// a, the source's reaction in r.  FIRST assigns a instead of adding.  POW: the
// pair function 1/r (1) or 1/r^2 (2), whose force is 2 r/r^4.
template <typename real, bool FORCES, int CK, bool FIRST, int POW>
__device__ __forceinline__ void nf_pair(const typename Vec4<real>::T &tv, int to, real sx, real sy, real sz,
                                        real sq, int so, real *a, real &rp, real &rx, real &ry, real &rz) {
    const real dx = tv.x - sx, dy = tv.y - sy, dz = tv.z - sz;
    const real r2 = dx * dx + dy * dy + dz * dz;
    real ri = rsqrt_pair<real>(r2);
    if (CK >= 1) ri = (so != to && (CK < 2 || r2 > real(0))) ? ri : real(0);
    const real pf = POW == 2 ? ri * ri : ri;  // the pair function
    if (FIRST) a[0] = sq * pf; else a[0] += sq * pf;
    rp += tv.w * pf;
    if (FORCES) {
        const real ri3 = POW == 2 ? real(2) * pf * pf : ri * ri * ri;  // |force| / (q q' r)
        const real as = sq * ri3, bt = tv.w * ri3;
        if (FIRST) {
            a[1] = as * dx;
            a[2] = as * dy;
            a[3] = as * dz;
        } else {
            a[1] += as * dx;
            a[2] += as * dy;
            a[3] += as * dz;
        }
        rx -= bt * dx;
        ry -= bt * dy;
        rz -= bt * dz;
    }
}

// Single precision, two targets at once: the pair (target 2q, source) in the
// low lane and (target 2q + 1, source) in the high lane of the packed FP32x2
// instructions (one issue slot for two pair evaluations).  ns*: the source
// position negated (d = t + ns = t - s); ntw: the targets' charges negated.
// The source's reaction accumulates as two partial sums, one per lane, with
// the sign of ntw (the potential's is flipped back at the end of the pass).
template <bool FORCES, int CK, bool FIRST, int POW>
__device__ __forceinline__ void nf_pair2(float2 tx, float2 ty, float2 tz, float2 ntw, int to0, int to1,
                                         float2 nsx, float2 nsy, float2 nsz, float2 sq, int so,
                                         float2 *a, float2 &rp, float2 &rx, float2 &ry, float2 &rz) {
    const float2 dx = __fadd2_rn(tx, nsx), dy = __fadd2_rn(ty, nsy), dz = __fadd2_rn(tz, nsz);
    const float2 r2 = __ffma2_rn(dz, dz, __ffma2_rn(dy, dy, __fmul2_rn(dx, dx)));
    float2 ri = make_float2(rsqrt_pair<float>(r2.x), rsqrt_pair<float>(r2.y));
    if (CK >= 1) {
        ri.x = (so != to0 && (CK < 2 || r2.x > 0.0f)) ? ri.x : 0.0f;
        ri.y = (so != to1 && (CK < 2 || r2.y > 0.0f)) ? ri.y : 0.0f;
    }
    const float2 pf = POW == 2 ? __fmul2_rn(ri, ri) : ri;  // the pair function
    if (FIRST) a[0] = __fmul2_rn(sq, pf); else a[0] = __ffma2_rn(sq, pf, a[0]);
    rp = __ffma2_rn(ntw, pf, rp);  // minus the reaction potential
    if (FORCES) {
        const float2 ri3 = POW == 2 ? __fmul2_rn(__fadd2_rn(pf, pf), pf) : __fmul2_rn(__fmul2_rn(ri, ri), ri);
        const float2 as = __fmul2_rn(sq, ri3), nbt = __fmul2_rn(ntw, ri3);
        if (FIRST) {
            a[1] = __fmul2_rn(as, dx);
            a[2] = __fmul2_rn(as, dy);
            a[3] = __fmul2_rn(as, dz);
        } else {
            a[1] = __ffma2_rn(as, dx, a[1]);
            a[2] = __ffma2_rn(as, dy, a[2]);
            a[3] = __ffma2_rn(as, dz, a[3]);
        }
        rx = __ffma2_rn(nbt, dx, rx);
        ry = __ffma2_rn(nbt, dy, ry);
        rz = __ffma2_rn(nbt, dz, rz);
    }
}

// target i of a block into the pair layout: component h = i % 2 of pair i / 2
__device__ __forceinline__ void nf_stage_pair(float4 *tpa, float4 *tpb, int2 *tpo, int i, float4 v, int o) {
    float *a = reinterpret_cast<float *>(tpa + i / 2), *b = reinterpret_cast<float *>(tpb + i / 2);
    const int h = i & 1;
    a[h] = v.x;
    a[2 + h] = v.y;
    b[h] = v.z;
    b[2 + h] = -v.w;
    reinterpret_cast<int *>(tpo + i / 2)[h] = o;
}
__device__ __forceinline__ void nf_stage_pair(double4 *, double4 *, int2 *, int, double4, int) {}

// NT targets from g0 (an even count) against this thread's first KV of KS sources, packed
// by target pairs; the sums are transposed through shared memory in
// pair-major order (value (q, c, h) at q*2*NC + 2c + h, target 2q + h, component
// c) and summed over the warp's lanes in order into wp.
template <bool FORCES, int CK, int POW, int NT, int KS, int KV = KS>
__device__ __forceinline__ void nf_targets2(const float4 *tpa, const float4 *tpb, const int2 *tpo, int g0, int nt,
                                            const float2 (&nsx)[KS], const float2 (&nsy)[KS],
                                            const float2 (&nsz)[KS], const float2 (&sq)[KS], const int (&so)[KS],
                                            float2 (&rp)[KS], float2 (&rx)[KS], float2 (&ry)[KS],
                                            float2 (&rz)[KS], float *tb_w, float *wp, int lane) {
    constexpr int NC = FORCES ? 4 : 1;
    float2 acc[NT / 2 * NC];
    // with forces 4 target pairs, unrolled whole; potential only 16, unrolled
    // by 4 (whole, they spill)
    constexpr int QU = FORCES ? NF_QUNROLL : (NF_QUNROLL < 4 ? NF_QUNROLL : 4);
#pragma unroll QU
    for (int q = 0; q < NT / 2; q++) {
        // target pair (g0 + 2q, g0 + 2q + 1): (x0, x1, y0, y1), (z0, z1, -w0, -w1)
        const float4 A = tpa[g0 / 2 + q], Bv = tpb[g0 / 2 + q];
        const int2 O = tpo[g0 / 2 + q];
        const float2 tx = make_float2(A.x, A.y), ty = make_float2(A.z, A.w), tz = make_float2(Bv.x, Bv.y);
        const float2 ntw = make_float2(Bv.z, Bv.w);
        nf_pair2<FORCES, CK, true, POW>(tx, ty, tz, ntw, O.x, O.y, nsx[0], nsy[0], nsz[0], sq[0], so[0],
                                        acc + q * NC, rp[0], rx[0], ry[0], rz[0]);
#pragma unroll
        for (int k = 1; k < KV; k++)
            nf_pair2<FORCES, CK, false, POW>(tx, ty, tz, ntw, O.x, O.y, nsx[k], nsy[k], nsz[k], sq[k], so[k],
                                             acc + q * NC, rp[k], rx[k], ry[k], rz[k]);
    }
    constexpr int NV = NT * NC;  // values per lane
    __syncwarp();
#pragma unroll
    for (int v = 0; v < NV / 2; v += 2)
        *reinterpret_cast<float4 *>(tb_w + lane * NF_TP + 2 * v) =
            make_float4(acc[v].x, acc[v].y, acc[v + 1].x, acc[v + 1].y);
    __syncwarp();
    if (lane < NV) {
        float tot = tb_w[lane];
#pragma unroll
        for (int r = 1; r < 32; r++) tot += tb_w[r * NF_TP + lane];
        const int q = lane / (2 * NC), c = (lane / 2) % NC, h = lane % 2;
        const int u = 2 * q + h;
        if (g0 + u < nt) wp[(g0 + u) * NC + c] = tot;
    }
}

template <typename real, bool FORCES, int CK, int POW>
struct KP2P {
    static constexpr int BS = NF_BS, MINB = sizeof(real) == 4 ? NF_MINB : 1;
    int depth;
    int periodic;
    const int *__restrict__ leaf_start;
    const typename Vec4<real>::T *__restrict__ s_pt;
    const int *__restrict__ s_origin;
    typename Vec4<real>::T *__restrict__ out_pt;
    typename Vec4<real>::T *__restrict__ react;
    int64_t rstride;
    const int *__restrict__ pord;
    __device__ __forceinline__ void run(const int bid_, const int nblk_) const {
        typedef typename Vec4<real>::T real4;
        constexpr int NC = FORCES ? 4 : 1;     // components per target
        constexpr int TG = 32 / NC;            // targets per transposed group
        constexpr int TR = FORCES ? 2 : 8;     // targets per remainder group
        constexpr int NW = NF_BS / 32;
        constexpr int NF_TB = sizeof(real) == 8 ? 64 : 256;
        __shared__ real4 tpos[NF_TB];
        __shared__ int tori[NF_TB];
        // single precision: the targets again by pairs, (x0, x1, y0, y1),
        // (z0, z1, -w0, -w1) and the two origins (the packed pair evaluations)
        constexpr int NPR = sizeof(real) == 4 ? NF_TB / 2 : 1;
        __shared__ float4 tpa[NPR], tpb[NPR];
        __shared__ int2 tpo[NPR];
        constexpr int WP = NF_TB * NC > 128 ? NF_TB * NC : 128;  // the own phase uses 128 per warp
        __shared__ real wpart[NW][WP];
        __shared__ __align__(16) real tbuf[NW][32 * NF_TP];
        // seg_off: prefix of the 13 forward segments' sizes, then sentinels up to
        // index 16 for the 4-step search of a slot's segment
        __shared__ int seg_start[NF_SEGS], seg_off[NF_SEGS + 3];

        // the cell of this CTA: the launch order's entry (occupied cells, heaviest
        // first), or the block index where there is no order (small grids)
        uint32_t key = bid_;
        if (pord) {
            int nocc = 0;
#pragma unroll
            for (int k = 0; k < NF_NCLS; k++) nocc += pord[k];
            if ((int)bid_ >= nocc) return;
            key = (uint32_t)pord[16 + bid_];
        }
        const int t0 = leaf_start[key], T = leaf_start[key + 1] - t0;
        if (T == 0) return;
        const int S = 1 << depth;
        int cx, cy, cz;
        morton_decode(key, cx, cy, cz);
        // a cell whose charges fit one target block stages them once, here, so that
        // their loads overlap the segment lookups (padded to a whole remainder
        // group with inert targets: far from every source, no charge, an origin no
        // source has)
        const bool one_block = T <= NF_TB;
        if (one_block) {
            const int ntp = (T + TR - 1) / TR * TR;
            for (int i = threadIdx.x; i < ntp; i += NF_BS) {
                real4 v;
                int o;
                if (i < T) {
                    v = s_pt[t0 + i];
                    o = s_origin[t0 + i];
                } else {
                    const real far = -(real)(4 * S + 16);
                    v = make_vec4(far, far, far, real(0));
                    o = -2;
                }
                tpos[i] = v;
                tori[i] = o;
                if constexpr (sizeof(real) == 4) nf_stage_pair(tpa, tpb, tpo, i, v, o);
            }
        }
        // forward segments d = 1..13 at [d - 1]: warp 0, sizes summed by a shuffle scan
        if (threadIdx.x < 32) {
            const int l = threadIdx.x;
            int st = 0, cnt = 0;
            if (l < NF_SEGS - 1) {
                int dx, dy, dz;
                nf_delta(l + 1, dx, dy, dz);
                const int64_t b = nf_cell(cx, cy, cz, dx, dy, dz, S, periodic);
                if (b >= 0) {
                    st = leaf_start[b];
                    cnt = leaf_start[b + 1] - st;
                }
                seg_start[l] = st;
            }
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, cnt, o);
                if (l >= o) cnt += v;
            }
            if (l == 0) seg_off[0] = 0;
            if (l < NF_SEGS - 1) seg_off[l + 1] = cnt;
            else if (l < NF_SEGS + 2) seg_off[l + 1] = 0x7fffffff;
        }
        __syncthreads();
        const int Ns = seg_off[NF_SEGS - 1];
        const int npass = (Ns + NF_BS * NF_KS - 1) / (NF_BS * NF_KS);
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const real Sr = (real)S;
        const real Sp = POW == 2 ? Sr * Sr : Sr;  // unit-box scale of the pair function
        real *tb_w = tbuf[warp];

        // ---- forward phase (mutual) ----
        for (int pass = 0; pass < npass; pass++) {
            real sx[NF_KS], sy[NF_KS], sz[NF_KS], sq[NF_KS];
            int so[NF_KS], sidx[NF_KS], sseg[NF_KS];
            real rp[NF_KS], rx[NF_KS], ry[NF_KS], rz[NF_KS];
#pragma unroll
            for (int k = 0; k < NF_KS; k++) {
                const int f = pass * NF_BS * NF_KS + k * NF_BS + threadIdx.x;
                // an empty slot: far away, no charge, origin that matches no target
                sx[k] = sy[k] = sz[k] = (real)(4 * S + 16);
                sq[k] = 0;
                so[k] = -1;
                sidx[k] = -1;
                sseg[k] = 0;
                rp[k] = rx[k] = ry[k] = rz[k] = 0;
                if (f < Ns) {
                    // the last segment starting at or before f (seg_off is non-decreasing)
                    int d = 0;
                    if (seg_off[d + 8] <= f) d += 8;
                    if (seg_off[d + 4] <= f) d += 4;
                    if (seg_off[d + 2] <= f) d += 2;
                    if (seg_off[d + 1] <= f) d += 1;
                    const int j = seg_start[d] + (f - seg_off[d]);
                    int dx, dy, dz;
                    nf_delta(d + 1, dx, dy, dz);
                    const real4 v = s_pt[j];
                    sx[k] = v.x + (real)dx;
                    sy[k] = v.y + (real)dy;
                    sz[k] = v.z + (real)dz;
                    sq[k] = v.w;
                    so[k] = s_origin[j];
                    sidx[k] = j;
                    sseg[k] = d;
                }
            }
            // single precision: the sources broadcast to both lanes of the packed
            // pair evaluations, positions negated; reactions as two partial sums
            float2 nsx2[NF_KS], nsy2[NF_KS], nsz2[NF_KS], sq2[NF_KS];
            float2 rp2[NF_KS], rx2[NF_KS], ry2[NF_KS], rz2[NF_KS];
            if constexpr (sizeof(real) == 4) {
#pragma unroll
                for (int k = 0; k < NF_KS; k++) {
                    nsx2[k] = make_float2(-sx[k], -sx[k]);
                    nsy2[k] = make_float2(-sy[k], -sy[k]);
                    nsz2[k] = make_float2(-sz[k], -sz[k]);
                    sq2[k] = make_float2(sq[k], sq[k]);
                    rp2[k] = rx2[k] = ry2[k] = rz2[k] = make_float2(0.0f, 0.0f);
                }
            }
            for (int tb = 0; tb < T; tb += NF_TB) {
                const int nt = min(NF_TB, T - tb);
                if (!one_block) {
                    __syncthreads();  // previous block's shared data consumed
                    // targets padded to a whole group with inert ones: far from every
                    // source, no charge, an origin no source has
                    // whole groups of TG, then the rest in groups of TR: pad to TR only
                    const int ntp = (nt + TR - 1) / TR * TR;
                    for (int i = threadIdx.x; i < ntp; i += NF_BS) {
                        real4 v;
                        int o;
                        if (i < nt) {
                            v = s_pt[t0 + tb + i];
                            o = s_origin[t0 + tb + i];
                        } else {
                            const real far = -(real)(4 * S + 16);
                            v = make_vec4(far, far, far, real(0));
                            o = -2;
                        }
                        tpos[i] = v;
                        tori[i] = o;
                        if constexpr (sizeof(real) == 4) nf_stage_pair(tpa, tpb, tpo, i, v, o);
                    }
                }
                // targets visible (staged before the prologue's barrier for one
                // block); the previous pass's reads of wpart done
                if (!one_block || pass > 0) __syncthreads();
                int g0 = 0;
                if constexpr (sizeof(real) == 4) {
                    // the source slots that hold a source in this pass (the same for
                    // the whole CTA: slot k of thread t is source k NF_BS + t)
                    const int rem = Ns - pass * NF_BS * NF_KS;
                    const int kv = rem <= NF_BS ? 1 : (rem <= 2 * NF_BS ? 2 : NF_KS);
#define NF_GROUPS(KV)                                                                                           \
    do {                                                                                                        \
        for (; g0 + TG <= nt; g0 += TG)                                                                         \
            nf_targets2<FORCES, CK, POW, TG, NF_KS, KV>(tpa, tpb, tpo, g0, nt, nsx2, nsy2, nsz2, sq2, so, rp2, rx2, \
                                                        ry2, rz2, tb_w, wpart[warp], lane);                     \
        for (; g0 < nt; g0 += TR)                                                                               \
            nf_targets2<FORCES, CK, POW, TR, NF_KS, KV>(tpa, tpb, tpo, g0, nt, nsx2, nsy2, nsz2, sq2, so, rp2, rx2, \
                                                        ry2, rz2, tb_w, wpart[warp], lane);                     \
    } while (0)
                    if (kv == 1) NF_GROUPS(1);
                    else if (kv == 2) NF_GROUPS(2);
                    else NF_GROUPS(NF_KS);
#undef NF_GROUPS
                }
                for (; g0 + TG <= nt; g0 += TG) {
                    real acc[32];
#pragma unroll
                    for (int u = 0; u < TG; u++) {
                        const real4 tv = tpos[g0 + u];
                        const int to = tori[g0 + u];
                        nf_pair<real, FORCES, CK, true, POW>(tv, to, sx[0], sy[0], sz[0], sq[0], so[0], acc + u * NC,
                                                           rp[0], rx[0], ry[0], rz[0]);
#pragma unroll
                        for (int k = 1; k < NF_KS; k++)
                            nf_pair<real, FORCES, CK, false, POW>(tv, to, sx[k], sy[k], sz[k], sq[k], so[k],
                                                                acc + u * NC, rp[k], rx[k], ry[k], rz[k]);
                    }
                    // transpose through shared memory: lane l sums value l over the lanes in order
                    __syncwarp();
#pragma unroll
                    for (int v = 0; v < 32; v += 4)
                        *reinterpret_cast<real4 *>(tb_w + lane * NF_TP + v) = make_vec4(acc[v], acc[v + 1], acc[v + 2], acc[v + 3]);
                    __syncwarp();
                    real tot = tb_w[lane];
#pragma unroll
                    for (int r = 1; r < 32; r++) tot += tb_w[r * NF_TP + lane];
                    if (g0 + lane / NC < nt) wpart[warp][(g0 + lane / NC) * NC + lane % NC] = tot;
                }
                for (; g0 < nt; g0 += TR) {  // the remaining targets, TR at a time
                    real acc[TR * NC];
#pragma unroll
                    for (int u = 0; u < TR; u++) {
                        const real4 tv = tpos[g0 + u];
                        const int to = tori[g0 + u];
                        nf_pair<real, FORCES, CK, true, POW>(tv, to, sx[0], sy[0], sz[0], sq[0], so[0], acc + u * NC,
                                                           rp[0], rx[0], ry[0], rz[0]);
#pragma unroll
                        for (int k = 1; k < NF_KS; k++)
                            nf_pair<real, FORCES, CK, false, POW>(tv, to, sx[k], sy[k], sz[k], sq[k], so[k],
                                                                acc + u * NC, rp[k], rx[k], ry[k], rz[k]);
                    }
                    __syncwarp();
#pragma unroll
                    for (int v = 0; v < TR * NC; v++) tb_w[lane * NF_TP + v] = acc[v];
                    __syncwarp();
                    if (lane < TR * NC) {
                        real tot = tb_w[lane];
#pragma unroll
                        for (int r = 1; r < 32; r++) tot += tb_w[r * NF_TP + lane];
                        if (g0 + lane / NC < nt) wpart[warp][(g0 + lane / NC) * NC + lane % NC] = tot;
                    }
                }
                __syncthreads();
                // target sums: the warps in order, then accumulated over passes; with
                // forces one thread per (target, component), all threads busy
                if (NC == 4) {
                    real *ob = reinterpret_cast<real *>(out_pt + t0 + tb);
                    for (int e = threadIdx.x; e < nt * 4; e += NF_BS) {
                        real t = wpart[0][e];
#pragma unroll
                        for (int w = 1; w < NW; w++) t += wpart[w][e];
                        if (pass > 0) t += ob[e];
                        ob[e] = t;
                    }
                } else
                for (int i = threadIdx.x; i < nt; i += NF_BS) {
                    real v[4] = {0, 0, 0, 0};
#pragma unroll
                    for (int c = 0; c < NC; c++) {
                        real t = wpart[0][i * NC + c];
#pragma unroll
                        for (int w = 1; w < NW; w++) t += wpart[w][i * NC + c];
                        v[c] = t;
                    }
                    real4 &o = out_pt[t0 + tb + i];
                    if (pass > 0) {
                        const real4 prev = o;
                        v[0] += prev.x;
                        v[1] += prev.y;
                        v[2] += prev.z;
                        v[3] += prev.w;
                    }
                    o = make_vec4(v[0], v[1], v[2], v[3]);
                }
            }
            if constexpr (sizeof(real) == 4) {
#pragma unroll
                for (int k = 0; k < NF_KS; k++) {
                    rp[k] = -(rp2[k].x + rp2[k].y);
                    rx[k] = rx2[k].x + rx2[k].y;
                    ry[k] = ry2[k].x + ry2[k].y;
                    rz[k] = rz2[k].x + rz2[k].y;
                }
            }
            // reactions of this pass's sources, complete after all target blocks;
            // unit-box units: 1/r_u^k = S^k/r_t^k, forces S^(k+1) times
#pragma unroll
            for (int k = 0; k < NF_KS; k++) {
                if (sidx[k] >= 0) {
                    const real qs = sq[k] * Sp * Sr;
                    react[sseg[k] * rstride + sidx[k]] = make_vec4(Sp * rp[k], qs * rx[k], qs * ry[k], qs * rz[k]);
                }
            }
        }

        // ---- own phase: pairs inside A, one-sided; a lane per target (chunks of
        // 32), the warps take every fourth source; warp partials summed in order ----
        // (one block: the cell's charges are still staged in tpos / tori and serve
        // as targets and sources; else sources are staged block by block in tbuf)
        real4 *spos = one_block ? tpos : reinterpret_cast<real4 *>(&tbuf[0][0]);
        int *sori = reinterpret_cast<int *>(&tori[0]);
        if (one_block) __syncthreads();  // the forward phase's reads of wpart done
        for (int c0 = 0; c0 < T; c0 += 32) {
            const int ti = c0 + lane;
            const bool act = ti < T;
            real4 tv = make_vec4(real(0), real(0), real(0), real(0));
            int to = -3;
            if (act) {
                tv = one_block ? tpos[ti] : s_pt[t0 + ti];
                to = one_block ? tori[ti] : s_origin[t0 + ti];
            }
            real pa = 0, xa = 0, ya = 0, za = 0;
            for (int sb = 0; sb < T; sb += NF_TB) {
                const int ns = min(NF_TB, T - sb);
                if (!one_block) {
                    __syncthreads();
                    for (int i = threadIdx.x; i < ns; i += NF_BS) {
                        spos[i] = s_pt[t0 + sb + i];
                        sori[i] = s_origin[t0 + sb + i];
                    }
                    __syncthreads();
                }
                if (act) {
#pragma unroll 4
                    for (int j = warp; j < ns; j += NW) {
                        const real4 sv = spos[j];
                        const real dx = tv.x - sv.x, dy = tv.y - sv.y, dz = tv.z - sv.z;
                        const real r2 = dx * dx + dy * dy + dz * dz;
                        real ri = rsqrt_pair<real>(r2);
                        ri = (r2 > real(0) && sori[j] != to) ? ri : real(0);
                        const real pf = POW == 2 ? ri * ri : ri;
                        pa += sv.w * pf;
                        if (FORCES) {
                            const real q3 = sv.w * (POW == 2 ? real(2) * pf * pf : ri * ri * ri);
                            xa += q3 * dx;
                            ya += q3 * dy;
                            za += q3 * dz;
                        }
                    }
                }
            }
            wpart[warp][lane * 4 + 0] = pa;
            wpart[warp][lane * 4 + 1] = xa;
            wpart[warp][lane * 4 + 2] = ya;
            wpart[warp][lane * 4 + 3] = za;
            __syncthreads();
            // A's own sums (forward phase + own pairs), scaled to unit-box units
            if (threadIdx.x < 32 && act) {
                real v[4];
#pragma unroll
                for (int c = 0; c < 4; c++) {
                    real t = wpart[0][lane * 4 + c];
#pragma unroll
                    for (int w = 1; w < NW; w++) t += wpart[w][lane * 4 + c];
                    v[c] = t;
                }
                real4 &o = out_pt[t0 + ti];
                if (npass > 0) {
                    const real4 prev = o;
                    v[0] += prev.x;
                    v[1] += prev.y;
                    v[2] += prev.z;
                    v[3] += prev.w;
                }
                const real qs = tv.w * Sp * Sr;
                o = make_vec4(Sp * v[0], qs * v[1], qs * v[2], qs * v[3]);
            }
            __syncthreads();
        }
    }
};
template <typename real, bool FORCES, int CK, int POW>
__global__ void __launch_bounds__(KP2P<real, FORCES, CK, POW>::BS, KP2P<real, FORCES, CK, POW>::MINB) k_p2p(const __grid_constant__ KP2P<real, FORCES, CK, POW> k) {
    k.run(blockIdx.x, gridDim.x);
}

template <typename real>
void launch_l2p(const Geom &g, const Coef<real> &C, const Ptrs<real> &P, const WsLayout &W,
                bool forces, cudaStream_t st, Tracer &tr) {
    const int ncell = (int)W.ncell, depth = g.depth;
    const real *loc_leaf = P.loc + W.loc_level[depth];
    const bool kf = forces && g.force_mode == FMM_FORCE_KERNEL;
    tr.begin(FMM_STAGE_L2P, st);
#define L2P(PP, F, K)                                                                              \
    launch_k(tr, FMM_TAG(S_L2P, 0), k_l2p<real, PP, F, K>,                                          \
             KL2P<real, PP, F, K>{C, depth, g.periodic, ncell, g.shift_free, P.leaf_start, P.s_pt, loc_leaf, \
                                  W.loc_comp, P.react, W.cap, P.out_pt, P.perm, P.out_e},            \
             (ncell + l2p_lpc<real, PP, K>() - 1) / l2p_lpc<real, PP, K>(), L2P_BS, 0, st)
    switch (g.p) {
#define CASE(PP)                                                                                 \
    case PP:                                                                                     \
        if (kf) L2P(PP, true, true);                                                             \
        else if (forces) L2P(PP, true, false);                                                   \
        else L2P(PP, false, false);                                                              \
        break;
        CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8)
#undef CASE
#undef L2P
    }
    tr.count();
    tr.end();
}

template <typename real>
void launch_p2p(const Geom &g, const Ptrs<real> &P, const WsLayout &W, bool forces,
                cudaStream_t st, Tracer &tr) {
    const int ncell = (int)W.ncell, depth = g.depth;
    tr.begin(FMM_STAGE_P2P, st);
    // pairs to skip (see k_p2p): none in the plain form; charges of the same
    // particle in the continuous form; also coincident charges there with odd p
    // (split charges on the cell plane)
    const int ck = !g.continuous ? 0 : ((g.p & 1) ? 2 : 1);
    // the launch order pays off where a few heavy cells could start late
    // among many light ones; grids of fewer than 32,768 cells go in cell order
    const int *pord = W.ncell >= 32768 ? P.pord : nullptr;
    if (pord) {
        zero_words(tr, FMM_TAG(S_ZERO_PORD, 0), P.pord, 16 * sizeof(int), st);
        const int nb = (int)((W.ncell + 255) / 256);
        launch_k(tr, FMM_TAG(S_NF_COUNT, 0), k_nf_order_count, KNfOrderCount{W.ncell, P.leaf_start, P.pord}, nb, 256,
                 0, st);
        tr.count();
        launch_k(tr, FMM_TAG(S_NF_FILL, 0), k_nf_order_fill, KNfOrderFill{W.ncell, P.leaf_start, P.pord}, nb, 256, 0,
                 st);
        tr.count();
    }
#define LAUNCH(F, CK)                                                                              \
    do {                                                                                           \
        if (g.power == 2)                                                                          \
            launch_k(tr, FMM_TAG(S_P2P, 0), k_p2p<real, F, CK, 2>,                                 \
                     KP2P<real, F, CK, 2>{depth, g.periodic, P.leaf_start, P.s_pt, P.s_origin, P.out_pt, \
                                          P.react, W.cap, pord},                                   \
                     ncell, NF_BS, 0, st);                                                         \
        else                                                                                       \
            launch_k(tr, FMM_TAG(S_P2P, 0), k_p2p<real, F, CK, 1>,                                 \
                     KP2P<real, F, CK, 1>{depth, g.periodic, P.leaf_start, P.s_pt, P.s_origin, P.out_pt, \
                                          P.react, W.cap, pord},                                   \
                     ncell, NF_BS, 0, st);                                                         \
    } while (0)
    if (forces) {
        if (ck == 2) LAUNCH(true, 2);
        else if (ck == 1) LAUNCH(true, 1);
        else LAUNCH(true, 0);
    } else {
        if (ck == 2) LAUNCH(false, 2);
        else if (ck == 1) LAUNCH(false, 1);
        else LAUNCH(false, 0);
    }
#undef LAUNCH
    tr.count();
    tr.end();
}

template void launch_l2p<float>(const Geom &, const Coef<float> &, const Ptrs<float> &,
                                const WsLayout &, bool, cudaStream_t, Tracer &);
template void launch_l2p<double>(const Geom &, const Coef<double> &, const Ptrs<double> &,
                                 const WsLayout &, bool, cudaStream_t, Tracer &);
template void launch_p2p<float>(const Geom &, const Ptrs<float> &, const WsLayout &, bool,
                                cudaStream_t, Tracer &);
template void launch_p2p<double>(const Geom &, const Ptrs<double> &, const WsLayout &, bool,
                                 cudaStream_t, Tracer &);

}  // namespace fmm

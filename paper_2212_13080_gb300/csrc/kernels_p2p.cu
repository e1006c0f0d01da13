// Evaluation at the charges: near field (step 5: direct sum over the finest
// cell and its 26 neighbours) and far field (§2.2 step 4 and the far-field force
// at the end of §2.2).  Results per sorted charge, unit-box units:
//   out_pt[slot] = (phi, F_x, F_y, F_z), phi per unit charge, F with the charge.
// The near-field kernel writes out_pt, the far-field kernel adds to it: the
// near field needs only the sorted charges and can run beside the far field.
#include "fmm_internal.cuh"
#include "lagrange.cuh"

namespace fmm {

__device__ __forceinline__ float4 make_vec4(float a, float b, float c, float d) { return make_float4(a, b, c, d); }
__device__ __forceinline__ double4 make_vec4(double a, double b, double c, double d) {
    return make_double4(a, b, c, d);
}

// ---------------------------------------------------------------------------
// far field: phi_far = sum_ijk g_i(t_x) g_j(t_y) g_k(t_z) L_leaf[ijk] and
// F_far = -q * 2^depth * grad_t phi_far.  One CTA per finest cell, L_leaf in
// shared memory, one thread per charge.
// ---------------------------------------------------------------------------
#define L2P_BS 64

template <typename real, int P, bool FORCES>
__global__ void __launch_bounds__(L2P_BS) k_l2p(Coef<real> C, int depth, const int *__restrict__ leaf_start,
                                                const typename Vec4<real>::T *__restrict__ s_pt,
                                                const real *__restrict__ loc_leaf,
                                                typename Vec4<real>::T *__restrict__ out_pt) {
    constexpr int P3 = P * P * P;
    __shared__ real Ls[P3];
    const uint32_t key = blockIdx.x;
    const int s0 = leaf_start[key], s1 = leaf_start[key + 1];
    if (s0 == s1) return;
    int cx, cy, cz;
    morton_decode(key, cx, cy, cz);
    const real *src = loc_leaf + loc_cell(depth, cx, cy, cz) * P3;
    for (int o = threadIdx.x; o < P3; o += blockDim.x) Ls[o] = src[o];
    __syncthreads();
    const real S = (real)(1 << depth);
    for (int s = s0 + threadIdx.x; s < s1; s += blockDim.x) {
        typename Vec4<real>::T v = s_pt[s];
        real gx[FMM_MAXP], gy[FMM_MAXP], gz[FMM_MAXP], dx[FMM_MAXP], dy[FMM_MAXP], dz[FMM_MAXP];
        if (FORCES) {
            lag_weights_deriv(C, P, v.x, gx, dx);
            lag_weights_deriv(C, P, v.y, gy, dy);
            lag_weights_deriv(C, P, v.z, gz, dz);
        } else {
            lag_weights(C, P, v.x, gx);
            lag_weights(C, P, v.y, gy);
            lag_weights(C, P, v.z, gz);
        }
        real phi = 0, fx = 0, fy = 0, fz = 0;
#pragma unroll 1
        for (int k = 0; k < P; k++) {
            real ax = 0, ay = 0, az = 0, aw = 0;
#pragma unroll
            for (int j = 0; j < P; j++) {
                real rx = 0, rdx = 0;
#pragma unroll
                for (int i = 0; i < P; i++) {
                    real Lv = Ls[(k * P + j) * P + i];
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
        typename Vec4<real>::T o = out_pt[s];  // the near field is already there
        o.x += phi;
        o.y += -v.w * S * fx;
        o.z += -v.w * S * fy;
        o.w += -v.w * S * fz;
        out_pt[s] = o;
    }
}

// ---------------------------------------------------------------------------
// near field.  One CTA of 128 threads per target cell.  The charges of the 27
// neighbour cells are staged in shared memory, shifted into the target cell's
// frame (source t + neighbour offset), in chunks.  Every thread owns two
// targets (one shared-memory source load serves two pairs); with T targets the
// CTA runs G = 128 / ceil(T/2) thread groups over the same targets, each taking
// every G-th source; the G partial sums are added in a fixed order.  Pairs of
// charges of the same particle (split charges) and coincident pairs are
// skipped.  Sums: blocks of up to 32 sources into a short partial, partials
// into the total with Kahan compensation.
// ---------------------------------------------------------------------------
template <typename real>
__device__ __forceinline__ void kahan_add(real &sum, real &c, real x) {
    real y = x - c;
    real t = sum + y;
    c = (t - sum) - y;
    sum = t;
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

template <typename real, bool FORCES>
struct PairAcc {
    real p, x, y, z;
    __device__ __forceinline__ void zero() { p = x = y = z = 0; }
    __device__ __forceinline__ void add(real tx, real ty, real tz, int to, const typename Vec4<real>::T &sv,
                                        int so) {
        real dx = tx - sv.x, dy = ty - sv.y, dz = tz - sv.z;
        real r2 = dx * dx + dy * dy + dz * dz;
        real ri = rsqrt_pair<real>(r2);
        ri = (r2 > real(0) && so != to) ? ri : real(0);
        real qr = sv.w * ri;
        p += qr;
        if (FORCES) {
            real qr3 = qr * (ri * ri);
            x += qr3 * dx;
            y += qr3 * dy;
            z += qr3 * dz;
        }
    }
};

#define P2P_BS 128
#define P2P_CHUNK 1024

template <typename real, bool FORCES>
__global__ void __launch_bounds__(P2P_BS) k_p2p(int depth, int periodic, const int *__restrict__ leaf_start,
                                                const typename Vec4<real>::T *__restrict__ s_pt,
                                                const int *__restrict__ s_origin,
                                                typename Vec4<real>::T *__restrict__ out_pt) {
    typedef typename Vec4<real>::T real4;
    __shared__ real4 src[P2P_CHUNK];
    __shared__ int srco[P2P_CHUNK];
    __shared__ int nb_start[27], nb_off[28];
    __shared__ real4 part[2 * P2P_BS];

    const uint32_t key = blockIdx.x;
    const int t0 = leaf_start[key], t1 = leaf_start[key + 1];
    const int T = t1 - t0;
    if (T == 0) return;
    const int S = 1 << depth;
    int cx, cy, cz;
    morton_decode(key, cx, cy, cz);
    if (threadIdx.x < 27) {
        int d = threadIdx.x;
        int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
        int nx = cx + dx, ny = cy + dy, nz = cz + dz;
        bool ok = true;
        if (periodic) {
            nx = (nx + S) % S;
            ny = (ny + S) % S;
            nz = (nz + S) % S;
        } else {
            ok = nx >= 0 && ny >= 0 && nz >= 0 && nx < S && ny < S && nz < S;
        }
        int st = 0, cnt = 0;
        if (ok) {
            uint32_t nk = morton_encode(nx, ny, nz);
            st = leaf_start[nk];
            cnt = leaf_start[nk + 1] - st;
        }
        nb_start[d] = st;
        nb_off[d + 1] = cnt;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        nb_off[0] = 0;
        for (int d = 0; d < 27; d++) nb_off[d + 1] += nb_off[d];
    }
    __syncthreads();
    const int Ns = nb_off[27];
    // thread -> (slot, group); a slot owns targets tb + slot and tb + TPP + slot
    int TPP, G;
    if (T >= 2 * P2P_BS) {
        TPP = P2P_BS;
        G = 1;
    } else {
        TPP = (T + 1) / 2;
        G = P2P_BS / TPP;
    }
    const int slot = threadIdx.x % TPP, grp = threadIdx.x / TPP;
    const bool grp_ok = grp < G;
    const bool single_chunk = Ns <= P2P_CHUNK;
    bool staged = false;
    const real S_r = (real)S;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    for (int tb = 0; tb < T; tb += 2 * TPP) {
        const int ta = tb + slot, tbb = tb + TPP + slot;
        const bool act_a = grp_ok && ta < T, act_b = grp_ok && tbb < T;
        real4 va, vb;
        int oa = -1, ob = -1;
        va.x = va.y = va.z = va.w = 0;
        vb = va;
        if (act_a) {
            va = s_pt[t0 + ta];
            oa = s_origin[t0 + ta];
        }
        if (act_b) {
            vb = s_pt[t0 + tbb];
            ob = s_origin[t0 + tbb];
        }
        PairAcc<real, FORCES> A, Bq, ca, cb;  // totals and Kahan compensations
        A.zero();
        Bq.zero();
        ca.zero();
        cb.zero();
        for (int c0 = 0; c0 < Ns; c0 += P2P_CHUNK) {
            const int cn = min(P2P_CHUNK, Ns - c0);
            if (!(single_chunk && staged)) {
                __syncthreads();
                // neighbour by neighbour, one warp per neighbour cell
                for (int d = warp; d < 27; d += P2P_BS / 32) {
                    const int lo = max(nb_off[d], c0), hi = min(nb_off[d + 1], c0 + cn);
                    const real ox = (real)(d % 3 - 1), oy = (real)((d / 3) % 3 - 1), oz = (real)(d / 9 - 1);
                    for (int f = lo + lane; f < hi; f += 32) {
                        const int sidx = nb_start[d] + f - nb_off[d];
                        real4 v = s_pt[sidx];
                        v.x += ox;
                        v.y += oy;
                        v.z += oz;
                        src[f - c0] = v;
                        srco[f - c0] = s_origin[sidx];
                    }
                }
                __syncthreads();
                staged = true;
            }
            if (act_a) {
                for (int sb = grp; sb < cn; sb += 32 * G) {
                    const int se = min(cn, sb + 32 * G);
                    PairAcc<real, FORCES> pa, pb;
                    pa.zero();
                    pb.zero();
#pragma unroll 4
                    for (int s = sb; s < se; s += G) {
                        const real4 sv = src[s];
                        const int so = srco[s];
                        pa.add(va.x, va.y, va.z, oa, sv, so);
                        pb.add(vb.x, vb.y, vb.z, ob, sv, so);
                    }
                    kahan_add(A.p, ca.p, pa.p);
                    kahan_add(Bq.p, cb.p, pb.p);
                    if (FORCES) {
                        kahan_add(A.x, ca.x, pa.x);
                        kahan_add(A.y, ca.y, pa.y);
                        kahan_add(A.z, ca.z, pa.z);
                        kahan_add(Bq.x, cb.x, pb.x);
                        kahan_add(Bq.y, cb.y, pb.y);
                        kahan_add(Bq.z, cb.z, pb.z);
                    }
                }
            }
        }
        // fixed-order sum over the groups, then add to the far field
        __syncthreads();
        part[threadIdx.x] = make_vec4(A.p, A.x, A.y, A.z);
        part[P2P_BS + threadIdx.x] = make_vec4(Bq.p, Bq.x, Bq.y, Bq.z);
        __syncthreads();
        for (int k = threadIdx.x; k < 2 * TPP; k += P2P_BS) {
            const int half = k / TPP, sl = k % TPP;
            const int tgt = tb + half * TPP + sl;
            if (tgt >= T) continue;
            real4 sum = part[half * P2P_BS + sl];
            for (int g2 = 1; g2 < G; g2++) {
                real4 o = part[half * P2P_BS + sl + g2 * TPP];
                sum.x += o.x;
                sum.y += o.y;
                sum.z += o.z;
                sum.w += o.w;
            }
            // unit-box units: 1/r_u = S / r_t, (x/r^3)_u = S^2 (x/r^3)_t
            const int si = t0 + tgt;
            const real qt = s_pt[si].w;
            out_pt[si] = make_vec4(S_r * sum.x, qt * S_r * S_r * sum.y, qt * S_r * S_r * sum.z,
                                   qt * S_r * S_r * sum.w);
        }
    }
}

template <typename real>
void launch_l2p(const Geom &g, const Coef<real> &C, const Ptrs<real> &P, const WsLayout &W,
                bool forces, cudaStream_t st, Tracer &tr) {
    const int ncell = (int)W.ncell, depth = g.depth;
    const real *loc_leaf = P.loc + W.loc_level[depth];
    tr.begin(FMM_STAGE_L2P, st);
    switch (g.p) {
#define CASE(PP)                                                                                 \
    case PP:                                                                                     \
        if (forces)                                                                              \
            k_l2p<real, PP, true><<<ncell, L2P_BS, 0, st>>>(C, depth, P.leaf_start, P.s_pt,     \
                                                           loc_leaf, P.out_pt);                 \
        else                                                                                     \
            k_l2p<real, PP, false><<<ncell, L2P_BS, 0, st>>>(C, depth, P.leaf_start, P.s_pt,    \
                                                            loc_leaf, P.out_pt);                \
        break;
        CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8)
#undef CASE
    }
    tr.count();
    tr.end();
}

template <typename real>
void launch_p2p(const Geom &g, const Ptrs<real> &P, const WsLayout &W, bool forces,
                cudaStream_t st, Tracer &tr) {
    const int ncell = (int)W.ncell, depth = g.depth;
    tr.begin(FMM_STAGE_P2P, st);
    if (forces)
        k_p2p<real, true><<<ncell, P2P_BS, 0, st>>>(depth, g.periodic, P.leaf_start, P.s_pt,
                                                    P.s_origin, P.out_pt);
    else
        k_p2p<real, false><<<ncell, P2P_BS, 0, st>>>(depth, g.periodic, P.leaf_start, P.s_pt,
                                                     P.s_origin, P.out_pt);
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

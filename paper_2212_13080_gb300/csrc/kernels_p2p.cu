// Evaluation at the charges: far field (§2.2 step 4 and the far-field force at
// the end of §2.2) and near field (step 5: direct sum over the finest cell and
// its 26 neighbours).  Results per sorted charge, unit-box units:
//   out_pt[slot] = (phi, F_x, F_y, F_z), phi per unit charge, F with the charge.
#include "fmm_internal.cuh"
#include "lagrange.cuh"

namespace fmm {

template <typename real> __device__ __forceinline__ real rsqrt_r(real x);
// single precision: the hardware reciprocal square root (2 ulp)
template <> __device__ __forceinline__ float rsqrt_r<float>(float x) { return rsqrtf(x); }
template <> __device__ __forceinline__ double rsqrt_r<double>(double x) { return 1.0 / sqrt(x); }

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
        typename Vec4<real>::T o;
        o.x = phi;
        o.y = -v.w * S * fx;
        o.z = -v.w * S * fy;
        o.w = -v.w * S * fz;
        out_pt[s] = o;
    }
}

// ---------------------------------------------------------------------------
// near field.  One CTA of 128 threads per target cell.  The charges of the 27
// neighbour cells are staged in shared memory, shifted into the target cell's
// frame (source t + neighbour offset), in chunks.  With T targets the CTA
// runs G = 128 / T thread groups over the same targets, each taking every
// G-th source; the G partial sums are added in a fixed order.  Pairs of charges
// of the same particle (split charges) and coincident pairs are skipped.
// ---------------------------------------------------------------------------
template <typename real>
__device__ __forceinline__ void kahan_add(real &sum, real &c, real x) {
    real y = x - c;
    real t = sum + y;
    c = (t - sum) - y;
    sum = t;
}

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
    __shared__ real nb_d[27][3];
    __shared__ real4 part[P2P_BS];

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
        nb_d[d][0] = (real)dx;
        nb_d[d][1] = (real)dy;
        nb_d[d][2] = (real)dz;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        nb_off[0] = 0;
        for (int d = 0; d < 27; d++) nb_off[d + 1] += nb_off[d];
    }
    __syncthreads();
    const int Ns = nb_off[27];
    int G, TPP;
    if (T >= P2P_BS) {
        G = 1;
        TPP = P2P_BS;
    } else {
        G = P2P_BS / T;
        TPP = T;
    }
    const int slot = threadIdx.x % TPP, grp = threadIdx.x / TPP;
    const bool grp_ok = grp < G;
    const bool single_chunk = Ns <= P2P_CHUNK;
    bool staged = false;
    const real S_r = (real)S;

    for (int tb = 0; tb < T; tb += TPP) {
        const int tgt = tb + slot;
        const bool active = grp_ok && tgt < T;
        real4 tv;
        int to = -1;
        if (active) {
            tv = s_pt[t0 + tgt];
            to = s_origin[t0 + tgt];
        } else {
            tv.x = tv.y = tv.z = tv.w = 0;
        }
        // totals with Kahan compensation; each block of up to 32 sources is
        // first summed into a short partial
        real phi = 0, fx = 0, fy = 0, fz = 0;
        real cphi = 0, cfx = 0, cfy = 0, cfz = 0;
        for (int c0 = 0; c0 < Ns; c0 += P2P_CHUNK) {
            const int cn = min(P2P_CHUNK, Ns - c0);
            if (!(single_chunk && staged)) {
                __syncthreads();
                for (int f = threadIdx.x; f < cn; f += P2P_BS) {
                    int ff = c0 + f;
                    int d = 0;
                    while (nb_off[d + 1] <= ff) d++;
                    int sidx = nb_start[d] + ff - nb_off[d];
                    real4 v = s_pt[sidx];
                    v.x += nb_d[d][0];
                    v.y += nb_d[d][1];
                    v.z += nb_d[d][2];
                    src[f] = v;
                    srco[f] = s_origin[sidx];
                }
                __syncthreads();
                staged = true;
            }
            if (active) {
                for (int sb = grp; sb < cn; sb += 32 * G) {
                    const int se = min(cn, sb + 32 * G);
                    real pp = 0, px = 0, py = 0, pz = 0;
                    for (int s = sb; s < se; s += G) {
                        real4 sv = src[s];
                        real dx = tv.x - sv.x, dy = tv.y - sv.y, dz = tv.z - sv.z;
                        real r2 = dx * dx + dy * dy + dz * dz;
                        bool ok = (r2 > real(0)) && (srco[s] != to);
                        real ri = ok ? rsqrt_r<real>(r2) : real(0);
                        real qr = sv.w * ri;
                        pp += qr;
                        if (FORCES) {
                            real qr3 = qr * ri * ri;
                            px += qr3 * dx;
                            py += qr3 * dy;
                            pz += qr3 * dz;
                        }
                    }
                    kahan_add(phi, cphi, pp);
                    if (FORCES) {
                        kahan_add(fx, cfx, px);
                        kahan_add(fy, cfy, py);
                        kahan_add(fz, cfz, pz);
                    }
                }
            }
        }
        // fixed-order sum over the groups, then add to the far field
        real4 pv;
        pv.x = phi;
        pv.y = fx;
        pv.z = fy;
        pv.w = fz;
        __syncthreads();
        part[threadIdx.x] = pv;
        __syncthreads();
        if (threadIdx.x < TPP && tb + threadIdx.x < T) {
            real4 s = part[threadIdx.x];
            for (int g2 = 1; g2 < G; g2++) {
                real4 o = part[threadIdx.x + g2 * TPP];
                s.x += o.x;
                s.y += o.y;
                s.z += o.z;
                s.w += o.w;
            }
            // unit-box units: 1/r_u = S / r_t, (x/r^3)_u = S^2 (x/r^3)_t
            const int sl = t0 + tb + threadIdx.x;
            real4 out = out_pt[sl];
            const real qt = s_pt[sl].w;
            out.x += S_r * s.x;
            out.y += qt * S_r * S_r * s.y;
            out.z += qt * S_r * S_r * s.z;
            out.w += qt * S_r * S_r * s.w;
            out_pt[sl] = out;
        }
    }
}

template <typename real>
void launch_evaluate(const Geom &g, const Coef<real> &C, const Ptrs<real> &P, const WsLayout &W,
                     bool forces, cudaStream_t st, Tracer &tr) {
    const int ncell = (int)W.ncell, depth = g.depth;
    const real *loc_leaf = P.loc + W.loc_level[depth];
    tr.begin(FMM_STAGE_L2P);
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
    tr.begin(FMM_STAGE_P2P);
    if (forces)
        k_p2p<real, true><<<ncell, P2P_BS, 0, st>>>(depth, g.periodic, P.leaf_start, P.s_pt,
                                                    P.s_origin, P.out_pt);
    else
        k_p2p<real, false><<<ncell, P2P_BS, 0, st>>>(depth, g.periodic, P.leaf_start, P.s_pt,
                                                     P.s_origin, P.out_pt);
    tr.count();
    tr.end();
}

template void launch_evaluate<float>(const Geom &, const Coef<float> &, const Ptrs<float> &,
                                     const WsLayout &, bool, cudaStream_t, Tracer &);
template void launch_evaluate<double>(const Geom &, const Coef<double> &, const Ptrs<double> &,
                                      const WsLayout &, bool, cudaStream_t, Tracer &);

}  // namespace fmm

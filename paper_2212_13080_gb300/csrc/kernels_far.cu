// Far field: replacement at the finest cells (P2M), shift up (M2M), the
// grid-to-grid bilinear forms of the interaction lists (M2L), the periodic
// lattice term, and the shift-transpose down (L2L).
#include <type_traits>

#include "fmm_internal.cuh"
#include "lagrange.cuh"

namespace fmm {

// ---------------------------------------------------------------------------
// §2.2 step 2, eq. (ex66): Phi_leaf[i,j,k] = sum_l q_l g_i(t_x) g_j(t_y) g_k(t_z).
// One CTA per finest cell.  A chunk of charges gets its 3p weights computed
// into shared memory, then every thread accumulates its grid nodes.
// ---------------------------------------------------------------------------
#define P2M_BS 128
#define P2M_CH 64

template <typename real, int P>
__global__ void __launch_bounds__(P2M_BS) k_p2m(Coef<real> C, int depth, const int *__restrict__ leaf_start,
                                                const typename Vec4<real>::T *__restrict__ s_pt,
                                                real *__restrict__ phi_leaf, real *__restrict__ q_leaf) {
    constexpr int P3 = P * P * P;
    __shared__ real wx[P2M_CH][P], wy[P2M_CH][P], wz[P2M_CH][P], wq[P2M_CH];
    const uint32_t key = blockIdx.x;
    int cx, cy, cz;
    morton_decode(key, cx, cy, cz);
    const int s0 = leaf_start[key], s1 = leaf_start[key + 1];
    constexpr int NO = (P3 + P2M_BS - 1) / P2M_BS;
    real acc[NO];
#pragma unroll
    for (int r = 0; r < NO; r++) acc[r] = 0;
    real Q = 0, Qc = 0;  // total charge of the cell (Kahan), thread 0
    for (int c0 = s0; c0 < s1; c0 += P2M_CH) {
        int m = min(P2M_CH, s1 - c0);
        if (threadIdx.x < m) {
            typename Vec4<real>::T v = s_pt[c0 + threadIdx.x];
            real g[FMM_MAXP];
            lag_weights(C, P, v.x, g);
#pragma unroll
            for (int i = 0; i < P; i++) wx[threadIdx.x][i] = g[i];
            lag_weights(C, P, v.y, g);
#pragma unroll
            for (int i = 0; i < P; i++) wy[threadIdx.x][i] = g[i];
            lag_weights(C, P, v.z, g);
#pragma unroll
            for (int i = 0; i < P; i++) wz[threadIdx.x][i] = g[i];
            wq[threadIdx.x] = v.w;
        }
        __syncthreads();
        if (threadIdx.x == 0)
            for (int t = 0; t < m; t++) {
                real y = wq[t] - Qc, tt = Q + y;
                Qc = (tt - Q) - y;
                Q = tt;
            }
#pragma unroll
        for (int r = 0; r < NO; r++) {
            int o = threadIdx.x + r * P2M_BS;
            if (o < P3) {
                int i = o % P, j = (o / P) % P, k = o / (P * P);
                real s = acc[r];
                for (int t = 0; t < m; t++) s += wq[t] * wx[t][i] * wy[t][j] * wz[t][k];
                acc[r] = s;
            }
        }
        __syncthreads();
    }
    const int64_t cell = phi_cell(depth, cx, cy, cz);
    real *out = phi_leaf + cell * P3;
#pragma unroll
    for (int r = 0; r < NO; r++) {
        int o = threadIdx.x + r * P2M_BS;
        if (o < P3) out[o] = acc[r];
    }
    if (threadIdx.x == 0) q_leaf[cell] = Q;
}

// ---------------------------------------------------------------------------
// §2.2 step 2, eq. (threethree): Phi_parent = sum_h (G_hx (x) G_hy (x) G_hz) Phi_child_h
// as three one-dimensional passes (x, y, z) over the 8 children in shared memory.
// One CTA per parent; children of level l, parent of level l-1.
// ---------------------------------------------------------------------------
#define M2M_BS 128

template <typename real>
__global__ void __launch_bounds__(M2M_BS) k_m2m(Coef<real> C, int p, int l, const real *__restrict__ phi_child,
                                                real *__restrict__ phi_parent,
                                                const real *__restrict__ q_child,
                                                real *__restrict__ q_parent) {
    extern __shared__ unsigned char smraw[];
    real *A = reinterpret_cast<real *>(smraw);
    const int p3 = p * p * p;
    real *B = A + 8 * p3;
    const int Hp = 1 << (l - 1);  // parents per axis
    const int pid = blockIdx.x;
    const int px = pid % Hp, py = (pid / Hp) % Hp, pz = pid / (Hp * Hp);
    for (int e = threadIdx.x; e < 8 * p3; e += blockDim.x) {
        int h = e / p3, o = e % p3;
        int cx = 2 * px + (h & 1), cy = 2 * py + ((h >> 1) & 1), cz = 2 * pz + (h >> 2);
        A[e] = phi_child[phi_cell(l, cx, cy, cz) * p3 + o];
    }
    __syncthreads();
    // x pass: B[h][k][j][I] = sum_i G_hx[I][i] A[h][k][j][i]
    for (int e = threadIdx.x; e < 8 * p3; e += blockDim.x) {
        int h = e / p3, o = e % p3, I = o % p, row = o - I;
        const real *G = C.G[h & 1];
        real s = 0;
        for (int i = 0; i < p; i++) s += G[I * p + i] * A[h * p3 + row + i];
        B[e] = s;
    }
    __syncthreads();
    // y pass: A[h][k][J][I] = sum_j G_hy[J][j] B[h][k][j][I]
    for (int e = threadIdx.x; e < 8 * p3; e += blockDim.x) {
        int h = e / p3, o = e % p3, I = o % p, J = (o / p) % p, k = o / (p * p);
        const real *G = C.G[(h >> 1) & 1];
        real s = 0;
        for (int j = 0; j < p; j++) s += G[J * p + j] * B[h * p3 + (k * p + j) * p + I];
        A[e] = s;
    }
    __syncthreads();
    // z pass and sum over the children
    real *out = phi_parent + phi_cell(l - 1, px, py, pz) * p3;
    for (int o = threadIdx.x; o < p3; o += blockDim.x) {
        int IJ = o % (p * p), K = o / (p * p);
        real s = 0;
        for (int h = 0; h < 8; h++) {
            const real *G = C.G[h >> 2];
            for (int k = 0; k < p; k++) s += G[K * p + k] * A[h * p3 + k * p * p + IJ];
        }
        out[o] = s;
    }
    if (threadIdx.x == 0) {
        real Q = 0;
        for (int h = 0; h < 8; h++)
            Q += q_child[phi_cell(l, 2 * px + (h & 1), 2 * py + ((h >> 1) & 1), 2 * pz + (h >> 2))];
        q_parent[phi_cell(l - 1, px, py, pz)] = Q;
    }
}

// Halo of the padded Phi layout of level l >= 1: open form zeros; periodic form
// the periodic image (coarse coordinate wrapped within the same parity block).
template <typename real>
__global__ void k_halo(int p3, int l, int periodic, real *__restrict__ phi_l, real *__restrict__ q_l) {
    const int H = 1 << (l - 1), P = H + 2;
    const int64_t ncells = 8LL * P * P * P;
    for (int64_t c = blockIdx.x; c < ncells; c += gridDim.x) {
        int X = (int)(c % P), Y = (int)((c / P) % P), Z = (int)((c / ((int64_t)P * P)) % P);
        int par = (int)(c / ((int64_t)P * P * P));
        bool shell = X == 0 || Y == 0 || Z == 0 || X == P - 1 || Y == P - 1 || Z == P - 1;
        if (!shell) continue;
        real *dst = phi_l + c * p3;
        if (!periodic) {
            for (int o = threadIdx.x; o < p3; o += blockDim.x) dst[o] = 0;
            if (threadIdx.x == 0) q_l[c] = 0;
        } else {
            int Xs = X == 0 ? H : (X == P - 1 ? 1 : X);
            int Ys = Y == 0 ? H : (Y == P - 1 ? 1 : Y);
            int Zs = Z == 0 ? H : (Z == P - 1 ? 1 : Z);
            const int64_t sc = (((int64_t)par * P + Zs) * P + Ys) * P + Xs;
            const real *src = phi_l + sc * p3;
            for (int o = threadIdx.x; o < p3; o += blockDim.x) dst[o] = src[o];
            if (threadIdx.x == 0) q_l[c] = q_l[sc];
        }
    }
}

// ---------------------------------------------------------------------------
// §2.2 step 3, eq. (bilinear): for every target cell C of level l and every C~ in
// its interaction list, L_C[a] += 2^l sum_b K_o[a,b] Phi_C~[b] with the unit-cell
// kernel K_o[a,b] = 1/|a - (o + b)|, o = C~ - C.  The interaction list of a cell of
// parity b (per axis) is the offsets o in [-2-b, 3-b]^3 without [-1,1]^3: 189.
//
// SIMT tiled contraction: one CTA per (tile of up to 4x4x4 target cells of one
// parity, chunk of 64 outputs a); per offset and per chunk of 64 inputs b the
// CTA stages the 64 source vectors (Ps[b][cell]) and K_o^T (Ks[b][a]; K_o^T =
// K_{-o}) in shared memory and every thread accumulates 4 cells x 4 outputs.
// Sources always lie inside the padded layout (halo), so no bounds checks.
// ---------------------------------------------------------------------------
#define M2L_BS 256
#define M2L_T 64

template <typename real>
__global__ void __launch_bounds__(M2L_BS) k_m2l_simt(int p, int l, const real *__restrict__ phi_l,
                                                     const real *__restrict__ q_l,
                                                     real *__restrict__ loc_l,
                                                     const real *__restrict__ KtT,
                                                     const real *__restrict__ Kbar, int ngroups) {
    typedef typename Vec4<real>::T real4;
    extern __shared__ __align__(16) unsigned char smraw[];
    real *Ps = reinterpret_cast<real *>(smraw);  // [64 b][64 cells]
    real *Ks = Ps + M2L_T * M2L_T;               // [64 b][64 a]
    real *Qs = Ks + M2L_T * M2L_T;               // [64 cells] source total charges
    real *Kb = Qs + M2L_T;                       // [64 a] row means
    const int p3 = p * p * p;
    const int H = 1 << (l - 1), P = H + 2;
    const int T = H < 4 ? H : 4;  // tile edge in coarse cells
    const int ntx = H / T;
    const int tile = blockIdx.x, par = blockIdx.y;
    const int a0 = (blockIdx.z / ngroups) * M2L_T, grp = blockIdx.z % ngroups;
    const int per = (189 + ngroups - 1) / ngroups;
    const int off_lo = grp * per, off_hi = off_lo + per;  // this CTA's offsets
    int off_idx = -1;
    const int TX = (tile % ntx) * T, TY = ((tile / ntx) % ntx) * T, TZ = (tile / (ntx * ntx)) * T;
    const int bx = par & 1, by = (par >> 1) & 1, bz = (par >> 2) & 1;
    const int ncell = T * T * T;
    const int cg = threadIdx.x / 16, ag = threadIdx.x % 16;
    // per-offset partial sums (64 terms) are added into the totals with Kahan
    // compensation: one FP32 accumulator over all 189 x 64 terms would lose
    // ~sqrt(12096/2) ulps
    real acc[4][4], tot[4][4], cmp[4][4];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) tot[i][j] = cmp[i][j] = 0;

    for (int oz = -2 - bz; oz <= 3 - bz; oz++)
        for (int oy = -2 - by; oy <= 3 - by; oy++)
            for (int ox = -2 - bx; ox <= 3 - bx; ox++) {
                if (ox >= -1 && ox <= 1 && oy >= -1 && oy <= 1 && oz >= -1 && oz <= 1) continue;
                off_idx++;
                if (off_idx < off_lo || off_idx >= off_hi) continue;
#pragma unroll
                for (int i = 0; i < 4; i++)
#pragma unroll
                    for (int j = 0; j < 4; j++) acc[i][j] = 0;
                // source parity and coarse shift
                const int sx = bx + ox, sy = by + oy, sz = bz + oz;
                const int spar = (sx & 1) | ((sy & 1) << 1) | ((sz & 1) << 2);
                const int dX = sx >> 1, dY = sy >> 1, dZ = sz >> 1;
                const int oi = ((oz + 3) * 7 + (oy + 3)) * 7 + (ox + 3);
                const real *Kt = KtT + (int64_t)oi * p3 * p3;
                // monopole part: Kbar_o[a] * Q_source (the previous offset's
                // readers of Qs/Kb must be done first)
                __syncthreads();
                if (threadIdx.x < M2L_T) {
                    int ci = threadIdx.x;
                    real v = 0;
                    if (ci < ncell) {
                        int tx = ci % T, ty = (ci / T) % T, tz = ci / (T * T);
                        int64_t cell = (((int64_t)spar * P + TZ + tz + 1 + dZ) * P + TY + ty + 1 + dY) * P +
                                       TX + tx + 1 + dX;
                        v = q_l[cell];
                    }
                    Qs[ci] = v;
                } else if (threadIdx.x < 2 * M2L_T) {
                    int a = threadIdx.x - M2L_T;
                    Kb[a] = (a0 + a < p3) ? Kbar[(int64_t)oi * p3 + a0 + a] : real(0);
                }
                for (int b0 = 0; b0 < p3; b0 += M2L_T) {
                    // stage sources: Ps[b][ci]
                    for (int e = threadIdx.x; e < M2L_T * M2L_T; e += M2L_BS) {
                        int ci = e % M2L_T, b = e / M2L_T;
                        real v = 0;
                        if (ci < ncell && b0 + b < p3) {
                            int tx = ci % T, ty = (ci / T) % T, tz = ci / (T * T);
                            int64_t cell = (((int64_t)spar * P + TZ + tz + 1 + dZ) * P + TY + ty + 1 + dY) * P +
                                           TX + tx + 1 + dX;
                            v = phi_l[cell * p3 + b0 + b];
                        }
                        Ps[b * M2L_T + ci] = v;
                    }
                    // stage Kt_o^T: Ks[b][a] = Kt_o[a0+a][b0+b]
                    for (int e = threadIdx.x; e < M2L_T * M2L_T; e += M2L_BS) {
                        int a = e % M2L_T, b = e / M2L_T;
                        real v = 0;
                        if (a0 + a < p3 && b0 + b < p3) v = Kt[(int64_t)(b0 + b) * p3 + a0 + a];
                        Ks[b * M2L_T + a] = v;
                    }
                    __syncthreads();
                    const int bn = min(M2L_T, p3 - b0);
                    for (int b = 0; b < bn; b++) {
                        real4 pv = *reinterpret_cast<const real4 *>(&Ps[b * M2L_T + cg * 4]);
                        real4 kv = *reinterpret_cast<const real4 *>(&Ks[b * M2L_T + ag * 4]);
                        real pc[4] = {pv.x, pv.y, pv.z, pv.w};
                        real kc[4] = {kv.x, kv.y, kv.z, kv.w};
#pragma unroll
                        for (int i = 0; i < 4; i++)
#pragma unroll
                            for (int j = 0; j < 4; j++) acc[i][j] += pc[i] * kc[j];
                    }
                    __syncthreads();
                }
#pragma unroll
                for (int i = 0; i < 4; i++)
#pragma unroll
                    for (int j = 0; j < 4; j++) {
                        acc[i][j] += Kb[ag * 4 + j] * Qs[cg * 4 + i];
                        real y = acc[i][j] - cmp[i][j];
                        real t = tot[i][j] + y;
                        cmp[i][j] = (t - tot[i][j]) - y;
                        tot[i][j] = t;
                    }
            }
    // ngroups > 1: loc_l is the partial buffer of this group (level layout)
    const real scale = (real)(1 << l);
    real *dst = loc_l + (int64_t)grp * ((int64_t)1 << (3 * l)) * p3;
#pragma unroll
    for (int i = 0; i < 4; i++) {
        int ci = cg * 4 + i;
        if (ci >= ncell) continue;
        int tx = ci % T, ty = (ci / T) % T, tz = ci / (T * T);
        int cx = 2 * (TX + tx) + bx, cy = 2 * (TY + ty) + by, cz = 2 * (TZ + tz) + bz;
        real *out = dst + loc_cell(l, cx, cy, cz) * p3;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            int a = a0 + ag * 4 + j;
            if (a < p3) out[a] = scale * tot[i][j];
        }
    }
}

// sum of the offset-group partials, in group order
template <typename real>
__global__ void k_m2l_reduce(int ngroups, int64_t n, const real *__restrict__ part,
                             real *__restrict__ loc_l) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        real s = 0;
        for (int g = 0; g < ngroups; g++) s += part[(int64_t)g * n + i];
        loc_l[i] = s;
    }
}

// §4.2 (periodic form): the box against its images beyond the 26 nearest,
// L_0 = K_lat Phi_0 (level 0, unit box).
template <typename real>
__global__ void k_lattice(int p3, const real *__restrict__ Klt, const real *__restrict__ Klbar,
                          const real *__restrict__ phi0, const real *__restrict__ q0,
                          real *__restrict__ loc0) {
    for (int a = threadIdx.x; a < p3; a += blockDim.x) {
        real s = 0;
        for (int b = 0; b < p3; b++) s += Klt[(int64_t)a * p3 + b] * phi0[b];
        loc0[a] = s + Klbar[a] * q0[0];
    }
}

// ---------------------------------------------------------------------------
// §2.2 step 3: Psi_child(v) = Psi_parent(shift_{child->parent}(v)), i.e.
// L_child_h += (G_hx (x) G_hy (x) G_hz)^T L_parent, as three passes (z, y, x).
// One CTA per parent of level l-1; adds to the 8 children of level l (which
// already hold their own interaction-list contributions).
// ---------------------------------------------------------------------------
template <typename real>
__global__ void __launch_bounds__(M2M_BS) k_l2l(Coef<real> C, int p, int l, const real *__restrict__ loc_parent,
                                                real *__restrict__ loc_child) {
    extern __shared__ unsigned char smraw[];
    real *Lp = reinterpret_cast<real *>(smraw);
    const int p3 = p * p * p;
    real *A = Lp + p3;       // [hz][k][J][I]      2 p3
    real *B = A + 2 * p3;    // [hz][hy][k][j][I]  4 p3
    const int Hp = 1 << (l - 1);  // parents per axis (level l-1)
    const int pid = blockIdx.x;
    const int px = pid % Hp, py = (pid / Hp) % Hp, pz = pid / (Hp * Hp);
    const real *src = loc_parent + loc_cell(l - 1, px, py, pz) * p3;
    for (int o = threadIdx.x; o < p3; o += blockDim.x) Lp[o] = src[o];
    __syncthreads();
    for (int e = threadIdx.x; e < 2 * p3; e += blockDim.x) {
        int hz = e / p3, o = e % p3, IJ = o % (p * p), k = o / (p * p);
        const real *G = C.G[hz];
        real s = 0;
        for (int K = 0; K < p; K++) s += G[K * p + k] * Lp[K * p * p + IJ];
        A[e] = s;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 4 * p3; e += blockDim.x) {
        int hh = e / p3, o = e % p3, I = o % p, j = (o / p) % p, k = o / (p * p);
        int hz = hh >> 1, hy = hh & 1;
        const real *G = C.G[hy];
        real s = 0;
        for (int J = 0; J < p; J++) s += G[J * p + j] * A[hz * p3 + (k * p + J) * p + I];
        B[e] = s;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 8 * p3; e += blockDim.x) {
        int h = e / p3, o = e % p3, i = o % p, row = o - i;
        int hx = h & 1, hy = (h >> 1) & 1, hz = h >> 2;
        const real *G = C.G[hx];
        const real *b = B + ((hz << 1) | hy) * p3 + row;
        real s = 0;
        for (int I = 0; I < p; I++) s += G[I * p + i] * b[I];
        int cx = 2 * px + hx, cy = 2 * py + hy, cz = 2 * pz + hz;
        loc_child[loc_cell(l, cx, cy, cz) * p3 + o] += s;
    }
}

// ---------------------------------------------------------------------------
template <typename real>
void launch_upward(const Geom &g, const Coef<real> &C, const Ptrs<real> &P, const WsLayout &W,
                   cudaStream_t st, Tracer &tr) {
    const int p = g.p, p3 = g.p3, depth = g.depth;
    real *phi_leaf = P.phi + W.phi_level[depth];
    const int ncell = (int)W.ncell;
    tr.begin(FMM_STAGE_P2M);
    switch (p) {
#define CASE(PP) \
    case PP:                                                                                     \
        k_p2m<real, PP><<<ncell, P2M_BS, 0, st>>>(C, depth, P.leaf_start, P.s_pt, phi_leaf,      \
                                                  P.qlev + W.q_level[depth]);                    \
        break;
        CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8)
#undef CASE
    }
    tr.count();
    tr.end();
    tr.begin(FMM_STAGE_M2M);
    const int lmin = g.periodic ? 0 : 2;
    for (int l = depth; l >= 1; l--) {
        int blocks = (int)(phi_level_cells(l) < 4096 ? phi_level_cells(l) : 4096);
        k_halo<real><<<blocks, 64, 0, st>>>(p3, l, g.periodic, P.phi + W.phi_level[l],
                                            P.qlev + W.q_level[l]);
        tr.count();
        if (l - 1 >= lmin) {
            int nparent = 1 << (3 * (l - 1));
            size_t sm = sizeof(real) * 16 * p3;
            k_m2m<real><<<nparent, M2M_BS, sm, st>>>(C, p, l, P.phi + W.phi_level[l],
                                                     P.phi + W.phi_level[l - 1],
                                                     P.qlev + W.q_level[l], P.qlev + W.q_level[l - 1]);
            tr.count();
        }
    }
    tr.end();
}

template <typename real>
int launch_downward(const Geom &g, const Coef<real> &C, const Ptrs<real> &P, const WsLayout &W,
                    const DevTables<real> &T, const Streams &S, Tracer &tr) {
    cudaStream_t st = S.main;
    const int p = g.p, p3 = g.p3, depth = g.depth;
    const int achunks = (p3 + M2L_T - 1) / M2L_T;
    const size_t sm_m2l = sizeof(real) * (2 * M2L_T * M2L_T + 2 * M2L_T);
    const size_t sm_l2l = sizeof(real) * 7 * p3;
    // 1. every level's own interaction-list contributions (they only need Phi):
    //    L_0 = lattice term (periodic), L_l = sum over the interaction list
    const int lstart = g.periodic ? 1 : 2;
    if (g.periodic) {
        tr.begin(FMM_STAGE_M2L);
        k_lattice<real><<<1, 256, 0, st>>>(p3, T.Klt, T.Klbar, P.phi + W.phi_level[0],
                                           P.qlev + W.q_level[0], P.loc + W.loc_level[0]);
        tr.count();
        tr.end();
    }
    int lsimt_end = depth;
    if (T.tc_lmin > 0 && depth >= T.tc_lmin) lsimt_end = T.tc_lmin - 1;
    // the SIMT levels run on the coarse stream, beside the tensor-core levels
    cudaEventRecord(S.fork, st);
    cudaStreamWaitEvent(S.coarse, S.fork, 0);
    for (int l = lstart; l <= lsimt_end; l++) {
        const int H = 1 << (l - 1);
        const int Tt = H < 4 ? H : 4;
        const int ntiles = (H / Tt) * (H / Tt) * (H / Tt);
        const int G = m2l_groups(l, p3);
        dim3 grid(ntiles, 8, achunks * G);
        real *dst = G > 1 ? P.m2l_part : P.loc + W.loc_level[l];
        tr.begin(FMM_STAGE_M2L, S.coarse);
        k_m2l_simt<real><<<grid, M2L_BS, sm_m2l, S.coarse>>>(p, l, P.phi + W.phi_level[l],
                                                             P.qlev + W.q_level[l], dst, T.KtT,
                                                             T.Kbar, G);
        tr.count();
        if (G > 1) {
            const int64_t n = ((int64_t)1 << (3 * l)) * p3;
            int nb = (int)((n + 255) / 256);
            if (nb > 152 * 16) nb = 152 * 16;
            k_m2l_reduce<real><<<nb, 256, 0, S.coarse>>>(G, n, P.m2l_part, P.loc + W.loc_level[l]);
            tr.count();
        }
        tr.end();
    }
    cudaEventRecord(S.coarse_done, S.coarse);
    if constexpr (std::is_same<real, float>::value) {
        if (T.tc_lmin > 0 && depth >= T.tc_lmin) {
            int rc = launch_m2l_tc(g, P, W, T.tc_khi_map, T.tc_klo_map, T.tc_kbar, T.tc_lmin,
                                   T.tc_mode, st, tr);
            if (rc) return rc;
        }
    }
    cudaStreamWaitEvent(st, S.coarse_done, 0);
    // 2. downward: Psi_child = Psi_parent o shift, added level by level
    for (int l = g.periodic ? 1 : 3; l <= depth; l++) {
        int nparent = 1 << (3 * (l - 1));
        tr.begin(FMM_STAGE_L2L);
        k_l2l<real><<<nparent, M2M_BS, sm_l2l, st>>>(C, p, l, P.loc + W.loc_level[l - 1],
                                                     P.loc + W.loc_level[l]);
        tr.count();
        tr.end();
    }
    return FMM_OK;
}

void far_set_attributes() {
    cudaFuncSetAttribute(k_m2l_simt<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 66 * 1024);
    cudaFuncSetAttribute(k_m2m<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 16 * 512 * 8);
    cudaFuncSetAttribute(k_m2m<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 16 * 512 * 4);
    cudaFuncSetAttribute(k_l2l<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 7 * 512 * 8);
    cudaFuncSetAttribute(k_l2l<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 7 * 512 * 4);
}

template void launch_upward<float>(const Geom &, const Coef<float> &, const Ptrs<float> &,
                                   const WsLayout &, cudaStream_t, Tracer &);
template void launch_upward<double>(const Geom &, const Coef<double> &, const Ptrs<double> &,
                                    const WsLayout &, cudaStream_t, Tracer &);
template int launch_downward<float>(const Geom &, const Coef<float> &, const Ptrs<float> &,
                                    const WsLayout &, const DevTables<float> &, const Streams &,
                                    Tracer &);
template int launch_downward<double>(const Geom &, const Coef<double> &, const Ptrs<double> &,
                                     const WsLayout &, const DevTables<double> &, const Streams &,
                                     Tracer &);

}  // namespace fmm

// Far field: replacement at the finest cells (P2M), shift up (M2M), the
// grid-to-grid bilinear forms of the interaction lists (M2L), the periodic
// lattice term, and the shift-transpose down (L2L).
#include <type_traits>

#include "fmm_internal.cuh"
#include "lagrange.cuh"
#include "launch.cuh"

namespace fmm {

// ---------------------------------------------------------------------------
// §2.2 step 2, eq. (ex66): Phi_leaf[i,j,k] = sum_l q_l g_i(t_x) g_j(t_y) g_k(t_z).
// One CTA per finest cell.  A chunk of charges gets its 3p weights computed
// into shared memory (x weights times the charge), then every thread
// accumulates its grid nodes; with p^3 < 128 the CTA runs 128 / p^3 thread
// groups over every G-th charge and adds their partials in a fixed order.  The
// cell's total charge: a warp tree per chunk, chunks added with compensation.
// ---------------------------------------------------------------------------
#define P2M_BS 128
#define P2M_CH 64

template <typename real, int P>
struct KP2M {
    static constexpr int BS = P2M_BS, MINB = 0;  // bounds on the block size only
    Coef<real> C;
    int depth;
    const int *__restrict__ leaf_start;
    const typename Vec4<real>::T *__restrict__ s_pt;
    real *__restrict__ phi_leaf;
    real *__restrict__ q_leaf;
    __device__ __forceinline__ void run(const int bid_, const int nblk_) const {
        constexpr int P3 = P * P * P;
        constexpr int G = P3 >= P2M_BS ? 1 : P2M_BS / P3;  // thread groups over the charges
        constexpr int NO = (P3 + P2M_BS - 1) / P2M_BS;     // nodes per thread (G == 1)
        __shared__ real wx[P2M_CH][P], wy[P2M_CH][P], wz[P2M_CH][P], wq[P2M_CH];
        __shared__ real part[G > 1 ? P2M_BS : 1];
        const uint32_t key = bid_;
        int cx, cy, cz;
        morton_decode(key, cx, cy, cz);
        const int s0 = leaf_start[key], s1 = leaf_start[key + 1];
        const int grp = G > 1 ? threadIdx.x / P3 : 0, node = G > 1 ? threadIdx.x % P3 : threadIdx.x;
        real acc[NO];
#pragma unroll
        for (int r = 0; r < NO; r++) acc[r] = 0;
        real Q = 0, Qc = 0;  // total charge of the cell (thread 0)
        for (int c0 = s0; c0 < s1; c0 += P2M_CH) {
            const int m = min(P2M_CH, s1 - c0);
            if (threadIdx.x < m) {
                typename Vec4<real>::T v = s_pt[c0 + threadIdx.x];
                real g[FMM_MAXP];
                lag_weights(C, P, v.x, g);
#pragma unroll
                for (int i = 0; i < P; i++) wx[threadIdx.x][i] = v.w * g[i];
                lag_weights(C, P, v.y, g);
#pragma unroll
                for (int i = 0; i < P; i++) wy[threadIdx.x][i] = g[i];
                lag_weights(C, P, v.z, g);
#pragma unroll
                for (int i = 0; i < P; i++) wz[threadIdx.x][i] = g[i];
                wq[threadIdx.x] = v.w;
            }
            __syncthreads();
            if (threadIdx.x < 32) {
                const int t = threadIdx.x;
                real v = (t < m ? wq[t] : real(0)) + (t + 32 < m ? wq[t + 32] : real(0));
                for (int o = 16; o >= 1; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
                if (t == 0) {
                    real y = v - Qc, tt = Q + y;
                    Qc = (tt - Q) - y;
                    Q = tt;
                }
            }
            if (grp < G) {
#pragma unroll
                for (int r = 0; r < NO; r++) {
                    const int o = node + r * P2M_BS;
                    if (o < P3) {
                        const int i = o % P, j = (o / P) % P, k = o / (P * P);
                        real s = acc[r];
                        for (int t = grp; t < m; t += G) s += wx[t][i] * wy[t][j] * wz[t][k];
                        acc[r] = s;
                    }
                }
            }
            __syncthreads();
        }
        const int64_t cell = phi_cell(depth, cx, cy, cz);
        real *out = phi_leaf + cell * P3;
        if (G > 1) {
            part[threadIdx.x] = grp < G ? acc[0] : real(0);
            __syncthreads();
            if (threadIdx.x < P3) {
                real s = part[threadIdx.x];
#pragma unroll
                for (int gi = 1; gi < G; gi++) s += part[gi * P3 + threadIdx.x];
                out[threadIdx.x] = s;
            }
        } else {
#pragma unroll
            for (int r = 0; r < NO; r++) {
                const int o = node + r * P2M_BS;
                if (o < P3) out[o] = acc[r];
            }
        }
        if (threadIdx.x == 0) q_leaf[cell] = Q;
    }
};
template <typename real, int P>
__global__ void __launch_bounds__(KP2M<real, P>::BS) k_p2m(const __grid_constant__ KP2M<real, P> k) {
    k.run(blockIdx.x, gridDim.x);
}

// Warp-per-cell form for p <= 6: four finest cells per CTA, one warp each,
// no block barriers (most finest cells of a non-uniform system are empty or
// light: a CTA per cell would spend its time on launch and barriers).  sf: the weights are taken at the box coordinate
// (c + t)/2^depth instead of the cell-local t (App. A.2, replacement with
// respect to the box).  Lane t computes the weights of the chunk's t-th charge
// into the warp's shared-memory rows; every lane then accumulates its grid
// nodes (lane, lane + 32, ...) over the chunk.  The cell's total charge: a warp
// tree per chunk, chunks added with compensation.
#ifndef P2M_WARPS
#define P2M_WARPS 4
#endif

template <typename real, int P>
struct KP2MWarp {
    static constexpr int BS = 32 * P2M_WARPS, MINB = 0;  // bounds on the block size only
    Coef<real> C;
    int depth;
    int ncell;
    int sf;
    const int *__restrict__ leaf_start;
    const typename Vec4<real>::T *__restrict__ s_pt;
    real *__restrict__ phi_leaf;
    real *__restrict__ q_leaf;
    __device__ __forceinline__ void run(const int bid_, const int nblk_) const {
        constexpr int P3 = P * P * P;
        constexpr int NO = (P3 + 31) / 32;
        __shared__ real w[P2M_WARPS][32][3 * P + 1];
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const int key = bid_ * P2M_WARPS + warp;
        if (key >= ncell) return;
        int cx, cy, cz;
        morton_decode((uint32_t)key, cx, cy, cz);
        const int s0 = leaf_start[key], s1 = leaf_start[key + 1];
        // coordinate of the weights: o + h t (cell-local: o = 0, h = 1)
        const real h = sf ? real(1) / (real)(1 << depth) : real(1);
        const real ox = sf ? h * cx : real(0), oy = sf ? h * cy : real(0), oz = sf ? h * cz : real(0);
        real (*ws)[3 * P + 1] = w[warp];
        real acc[NO];
#pragma unroll
        for (int r = 0; r < NO; r++) acc[r] = 0;
        real Q = 0, Qc = 0;
        for (int c0 = s0; c0 < s1; c0 += 32) {
            const int m = min(32, s1 - c0);
            real qv = 0;
            if (lane < m) {
                typename Vec4<real>::T v = s_pt[c0 + lane];
                real g[FMM_MAXP];
                lag_weights(C, P, ox + h * v.x, g);
#pragma unroll
                for (int i = 0; i < P; i++) ws[lane][i] = v.w * g[i];
                lag_weights(C, P, oy + h * v.y, g);
#pragma unroll
                for (int i = 0; i < P; i++) ws[lane][P + i] = g[i];
                lag_weights(C, P, oz + h * v.z, g);
#pragma unroll
                for (int i = 0; i < P; i++) ws[lane][2 * P + i] = g[i];
                qv = v.w;
            }
            for (int o = 16; o >= 1; o >>= 1) qv += __shfl_down_sync(0xffffffffu, qv, o);
            if (lane == 0) {
                real y = qv - Qc, tt = Q + y;
                Qc = (tt - Q) - y;
                Q = tt;
            }
            __syncwarp();
#pragma unroll
            for (int r = 0; r < NO; r++) {
                const int o = lane + 32 * r;
                if (o < P3) {
                    const int i = o % P, j = (o / P) % P, k = o / (P * P);
                    real sum = acc[r];
                    for (int t = 0; t < m; t++) sum += ws[t][i] * ws[t][P + j] * ws[t][2 * P + k];
                    acc[r] = sum;
                }
            }
            __syncwarp();
        }
        const int64_t cell = phi_cell(depth, cx, cy, cz);
        real *out = phi_leaf + cell * P3;
#pragma unroll
        for (int r = 0; r < NO; r++) {
            const int o = lane + 32 * r;
            if (o < P3) out[o] = acc[r];
        }
        if (lane == 0) q_leaf[cell] = Q;
    }
};
template <typename real, int P>
__global__ void __launch_bounds__(KP2MWarp<real, P>::BS) k_p2m_warp(const __grid_constant__ KP2MWarp<real, P> k) {
    k.run(blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------------
// §2.2 step 2, eq. (threethree): Phi_parent = sum_h (G_hx (x) G_hy (x) G_hz) Phi_child_h
// in the factored order: the x shift summed over the two x siblings (4 arrays),
// then the y shift summed over y (2 arrays), then z (1): 14 p^4 multiply-adds.
// One CTA per parent; children of level l, parent of level l-1.  p is a
// compile-time constant; the shift matrices are staged in shared memory.
// ---------------------------------------------------------------------------
#define M2M_BS 128

template <typename real, int P>
struct KM2M {
    static constexpr int BS = M2M_BS, MINB = 0;  // bounds on the block size only
    Coef<real> C;
    int l;
    const real *__restrict__ phi_child;
    real *__restrict__ phi_parent;
    const real *__restrict__ q_child;
    real *__restrict__ q_parent;
    int depth;
    const int *__restrict__ leaf_start;
    __device__ __forceinline__ void run(const int bid_, const int nblk_) const {
        constexpr int P3 = P * P * P, PP = P * P;
        extern __shared__ unsigned char smraw[];
        real *A = reinterpret_cast<real *>(smraw);  // [h][k][j][i]          8 p^3
        real *B = A + 8 * P3;                       // [hz][hy][k][j][I]     4 p^3
        real *D = B + 4 * P3;                       // [hz][k][J][I]         2 p^3
        real *Gs = D + 2 * P3;                      // [h][J][i]             2 p^2
        const int Hp = 1 << (l - 1);                // parents per axis
        const int pid = bid_;
        const int px = pid % Hp, py = (pid / Hp) % Hp, pz = pid / (Hp * Hp);
        if (!cell_occupied(leaf_start, depth, l - 1, morton_encode(px, py, pz))) {
            // no charges below this parent: its children's grid charges are all
            // zero, and so are its own (what the sums below give)
            real *out = phi_parent + phi_cell(l - 1, px, py, pz) * P3;
            for (int o = threadIdx.x; o < P3; o += M2M_BS) out[o] = real(0);
            if (threadIdx.x == 0) q_parent[phi_cell(l - 1, px, py, pz)] = real(0);
            return;
        }
        for (int e = threadIdx.x; e < 2 * PP; e += M2M_BS) Gs[e] = C.G[e / PP][e % PP];
        for (int e = threadIdx.x; e < 8 * P3; e += M2M_BS) {
            const int h = e / P3, o = e % P3;
            const int cx = 2 * px + (h & 1), cy = 2 * py + ((h >> 1) & 1), cz = 2 * pz + (h >> 2);
            A[e] = phi_child[phi_cell(l, cx, cy, cz) * P3 + o];
        }
        __syncthreads();
        for (int e = threadIdx.x; e < 4 * P3; e += M2M_BS) {
            const int hyz = e / P3, o = e % P3, I = o % P, row = o - I;
            real s = 0;
#pragma unroll
            for (int hx = 0; hx < 2; hx++) {
                const real *a = A + (hx + 2 * hyz) * P3 + row;
                const real *g = Gs + hx * PP + I * P;
#pragma unroll
                for (int i = 0; i < P; i++) s += g[i] * a[i];
            }
            B[e] = s;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < 2 * P3; e += M2M_BS) {
            const int hz = e / P3, o = e % P3, I = o % P, J = (o / P) % P, k = o / PP;
            real s = 0;
#pragma unroll
            for (int hy = 0; hy < 2; hy++) {
                const real *b = B + (hy + 2 * hz) * P3 + k * PP + I;
                const real *g = Gs + hy * PP + J * P;
#pragma unroll
                for (int j = 0; j < P; j++) s += g[j] * b[j * P];
            }
            D[e] = s;
        }
        __syncthreads();
        real *out = phi_parent + phi_cell(l - 1, px, py, pz) * P3;
        for (int o = threadIdx.x; o < P3; o += M2M_BS) {
            const int K = o / PP, IJ = o % PP;
            real s = 0;
#pragma unroll
            for (int hz = 0; hz < 2; hz++) {
                const real *d = D + hz * P3 + IJ;
                const real *g = Gs + hz * PP + K * P;
#pragma unroll
                for (int k = 0; k < P; k++) s += g[k] * d[k * PP];
            }
            out[o] = s;
        }
        if (threadIdx.x < 32) {  // total charge: the eight children, tree order
            real v = 0;
            if (threadIdx.x < 8) {
                const int h = threadIdx.x;
                v = q_child[phi_cell(l, 2 * px + (h & 1), 2 * py + ((h >> 1) & 1), 2 * pz + (h >> 2))];
            }
            for (int m = 4; m >= 1; m >>= 1) v += __shfl_down_sync(0xffffffffu, v, m);
            if (threadIdx.x == 0) q_parent[phi_cell(l - 1, px, py, pz)] = v;
        }
    }
};
template <typename real, int P>
__global__ void __launch_bounds__(KM2M<real, P>::BS) k_m2m(const __grid_constant__ KM2M<real, P> k) {
    k.run(blockIdx.x, gridDim.x);
}

template <typename real, int P>
constexpr size_t m2m_smem() {
    return sizeof(real) * (14 * P * P * P + 2 * P * P);
}

// Halo of the padded Phi layout of level l >= 1: open form zeros; periodic form
// the periodic image (coarse coordinate wrapped within the same parity block).
// One warp per (parity, Z, Y) row of the padded grid: a row on the y/z shell is
// all halo, any other row has its two x ends.
struct KHalo {
    static constexpr int BS = 0, MINB = 0;
    int p3;
    int l;
    int periodic;
    float *__restrict__ phi_f;
    double *__restrict__ phi_d;
    float *__restrict__ q_f;
    double *__restrict__ q_d;
    __device__ __forceinline__ void run(const int bid_, const int nblk_) const {
        const int H = 1 << (l - 1), P = H + 2;
        const int64_t nrows = 8LL * P * P;
        const int lane = threadIdx.x & 31;
        const int64_t w0 = (bid_ * (int64_t)blockDim.x + threadIdx.x) >> 5;
        const int64_t nw = ((int64_t)nblk_ * blockDim.x) >> 5;
        for (int64_t row = w0; row < nrows; row += nw) {
            const int Y = (int)(row % P), Z = (int)((row / P) % P);
            const int par = (int)(row / ((int64_t)P * P));
            const bool full = Y == 0 || Z == 0 || Y == P - 1 || Z == P - 1;
            const int ncell = full ? P : 2;
            for (int c = 0; c < ncell; c++) {
                const int X = full ? c : (c == 0 ? 0 : P - 1);
                const int64_t cell = ((int64_t)(par * P + Z) * P + Y) * P + X;
                int64_t sc = -1;
                if (periodic) {
                    const int Xs = X == 0 ? H : (X == P - 1 ? 1 : X);
                    const int Ys = Y == 0 ? H : (Y == P - 1 ? 1 : Y);
                    const int Zs = Z == 0 ? H : (Z == P - 1 ? 1 : Z);
                    sc = ((int64_t)(par * P + Zs) * P + Ys) * P + Xs;
                }
                if (phi_f) {
                    for (int o = lane; o < p3; o += 32) phi_f[cell * p3 + o] = sc >= 0 ? phi_f[sc * p3 + o] : 0.0f;
                    if (lane == 0) q_f[cell] = sc >= 0 ? q_f[sc] : 0.0f;
                } else {
                    for (int o = lane; o < p3; o += 32) phi_d[cell * p3 + o] = sc >= 0 ? phi_d[sc * p3 + o] : 0.0;
                    if (lane == 0) q_d[cell] = sc >= 0 ? q_d[sc] : 0.0;
                }
            }
        }
    }
};
__global__ void k_halo_rows(const __grid_constant__ KHalo k) {
    k.run(blockIdx.x, gridDim.x);
}

template <typename real>
void launch_halo(int p3, int l, int periodic, real *phi_l, real *q_l, cudaStream_t st, Tracer &tr) {
    const int P = (1 << (l - 1)) + 2;
    const int64_t nrows = 8LL * P * P;
    int blocks = (int)((nrows * 32 + 255) / 256);
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (std::is_same<real, float>::value)
        launch_k(tr, FMM_TAG(S_HALO, l), k_halo_rows,
                 KHalo{p3, l, periodic, (float *)phi_l, nullptr, (float *)q_l, nullptr}, blocks, 256, 0, st);
    else
        launch_k(tr, FMM_TAG(S_HALO, l), k_halo_rows,
                 KHalo{p3, l, periodic, nullptr, (double *)phi_l, nullptr, (double *)q_l}, blocks, 256, 0, st);
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
#define M2L_PS (M2L_T + 4)  // row stride of the staged source values (keeps rows 16-byte aligned)

template <typename real>
struct KM2LSimt {
    static constexpr int BS = M2L_BS, MINB = sizeof(real) == 4 ? 2 : 0;  // FP32: two CTAs per SM
    int p;
    int l;
    const real *__restrict__ phi_l;
    const real *__restrict__ q_l;
    real *__restrict__ loc_l;
    const real *__restrict__ KtT;
    const real *__restrict__ Kbar;
    int ngroups;
    int spow;
    int ntiles;  // grid: tile fastest, then the 8 parities, then a-chunk x group
    const int *__restrict__ leaf_start;  // target cells' occupancy (finest level depth)
    int depth;
    __device__ __forceinline__ void run(const int bid_, const int nblk_) const {
        typedef typename Vec4<real>::T real4;
        extern __shared__ __align__(16) unsigned char smraw[];
        real *Ps = reinterpret_cast<real *>(smraw);  // [64 cells][M2L_PS]: b fastest
        real *Ks = Ps + M2L_T * M2L_PS;              // [64 b][64 a]
        real *Qs = Ks + M2L_T * M2L_T;               // [64 cells] source total charges
        real *Kb = Qs + M2L_T;                       // [64 a] row means
        const int p3 = p * p * p;
        const int H = 1 << (l - 1), P = H + 2;
        const int T = H < 4 ? H : 4;  // tile edge in coarse cells
        const int ntx = H / T;
        const int tile = bid_ % ntiles, par = (bid_ / ntiles) % 8, zg = bid_ / (ntiles * 8);
        const int a0 = (zg / ngroups) * M2L_T, grp = zg % ngroups;
        const int per = (189 + ngroups - 1) / ngroups;
        const int off_lo = grp * per, off_hi = off_lo + per;  // this CTA's offsets
        int off_idx = -1;
        const int TX = (tile % ntx) * T, TY = ((tile / ntx) % ntx) * T, TZ = (tile / (ntx * ntx)) * T;
        const int bx = par & 1, by = (par >> 1) & 1, bz = (par >> 2) & 1;
        const int ncell = T * T * T;
        // a tile none of whose target cells holds a charge forms no functional
        // that is read (step 4 reads the functionals of occupied cells only)
        {
            int occ = 0;
            if ((int)threadIdx.x < ncell) {
                const int ci = threadIdx.x, tx = ci % T, ty = (ci / T) % T, tz = ci / (T * T);
                const uint32_t key = morton_encode(2 * (TX + tx) + bx, 2 * (TY + ty) + by, 2 * (TZ + tz) + bz);
                occ = cell_occupied(leaf_start, depth, l, key);
            }
            if (!__syncthreads_or(occ)) return;
        }
        const int cg = threadIdx.x / 16, ag = threadIdx.x % 16;
        // the cells this thread stages: value b = threadIdx % 64 of cells
        // c = threadIdx / 64 + 4 it; with T = 4, cell c of the tile is
        // (c % 4, c / 4 % 4, c / 16): x = threadIdx / 64, y = it % 4, z = it / 4
        const int c0 = (int)threadIdx.x / M2L_T;
        const int rb = ((TZ + 1) * P + TY + 1) * P + TX + c0 + 1;
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
                    const int64_t sbase = (int64_t)spar * P * P * P + ((int64_t)dZ * P + dY) * P + dX;
                    for (int b0 = 0; b0 < p3; b0 += M2L_T) {
                        // stage sources: Ps[ci][b], b fastest (coalesced reads of a cell's values)
                        const int b = threadIdx.x % M2L_T;
#pragma unroll
                        for (int it = 0; it < M2L_T * M2L_T / M2L_BS; it++) {
                            const int ci = c0 + (M2L_BS / M2L_T) * it;
                            int r;
                            if (T == 4) {
                                r = rb + ((it >> 2) * P + (it & 3)) * P;
                            } else {
                                const int tx = ci % T, ty = (ci / T) % T, tz = ci / (T * T);
                                r = ci < ncell ? ((TZ + tz + 1) * P + TY + ty + 1) * P + TX + tx + 1 : -1;
                            }
                            real v = 0;
                            if (r >= 0 && b0 + b < p3) v = phi_l[(sbase + r) * p3 + b0 + b];
                            Ps[ci * M2L_PS + b] = v;
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
                        int bb = 0;
                        for (; bb + 4 <= bn; bb += 4) {  // four values b of four cells per load
                            real pv[4][4];
#pragma unroll
                            for (int i = 0; i < 4; i++) {
                                const real4 v = *reinterpret_cast<const real4 *>(&Ps[(cg * 4 + i) * M2L_PS + bb]);
                                pv[i][0] = v.x;
                                pv[i][1] = v.y;
                                pv[i][2] = v.z;
                                pv[i][3] = v.w;
                            }
#pragma unroll
                            for (int u = 0; u < 4; u++) {
                                const real4 kv = *reinterpret_cast<const real4 *>(&Ks[(bb + u) * M2L_T + ag * 4]);
                                const real kc[4] = {kv.x, kv.y, kv.z, kv.w};
#pragma unroll
                                for (int i = 0; i < 4; i++)
#pragma unroll
                                    for (int j = 0; j < 4; j++) acc[i][j] += pv[i][u] * kc[j];
                            }
                        }
                        for (; bb < bn; bb++) {
                            const real4 kv = *reinterpret_cast<const real4 *>(&Ks[bb * M2L_T + ag * 4]);
                            const real kc[4] = {kv.x, kv.y, kv.z, kv.w};
#pragma unroll
                            for (int i = 0; i < 4; i++) {
                                const real pc = Ps[(cg * 4 + i) * M2L_PS + bb];
#pragma unroll
                                for (int j = 0; j < 4; j++) acc[i][j] += pc * kc[j];
                            }
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
        const real scale = (real)(1 << (l * spow));  // unit cells -> unit box: 2^l (1/r), 4^l (r/|r|^3)
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
};
template <typename real>
__global__ void __launch_bounds__(KM2LSimt<real>::BS, sizeof(real) == 4 ? 2 : 1) k_m2l_simt(const __grid_constant__ KM2LSimt<real> k) {
    k.run(blockIdx.x, gridDim.x);
}

// sum of the offset-group partials, in group order
template <typename real>
struct KM2LReduce {
    static constexpr int BS = 0, MINB = 0;
    int ngroups;
    int64_t n;
    const real *__restrict__ part;
    real *__restrict__ loc_l;
    __device__ __forceinline__ void run(const int bid_, const int nblk_) const {
        for (int64_t i = bid_ * (int64_t)blockDim.x + threadIdx.x; i < n;
             i += (int64_t)nblk_ * blockDim.x) {
            real s = 0;
            for (int g = 0; g < ngroups; g++) s += part[(int64_t)g * n + i];
            loc_l[i] = s;
        }
    }
};
template <typename real>
__global__ void k_m2l_reduce(const __grid_constant__ KM2LReduce<real> k) {
    k.run(blockIdx.x, gridDim.x);
}

// §4.2 (periodic form): the box against its images beyond the 26 nearest,
// L_0 = K_lat Phi_0 (level 0, unit box).
template <typename real>
struct KLattice {
    static constexpr int BS = 0, MINB = 0;
    int p3;
    const real *__restrict__ Klt;
    const real *__restrict__ Klbar;
    const real *__restrict__ phi0;
    const real *__restrict__ q0;
    real *__restrict__ loc0;
    __device__ __forceinline__ void run(const int bid_, const int nblk_) const {
        for (int a = threadIdx.x; a < p3; a += blockDim.x) {
            real s = 0;
            for (int b = 0; b < p3; b++) s += Klt[(int64_t)a * p3 + b] * phi0[b];
            loc0[a] = s + Klbar[a] * q0[0];
        }
    }
};
template <typename real>
__global__ void k_lattice(const __grid_constant__ KLattice<real> k) {
    k.run(blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------------
// §2.2 step 3: Psi_child(v) = Psi_parent(shift_{child->parent}(v)), i.e.
// L_child_h += (G_hx (x) G_hy (x) G_hz)^T L_parent, as three passes (z, y, x).
// One CTA per parent of level l-1; adds to the 8 children of level l (which
// already hold their own interaction-list contributions).  Only cells that
// hold charges are formed: step 4 reads no other functional, and the children
// of a cell without charges hold none either.
// ---------------------------------------------------------------------------
template <typename real, int P>
struct KL2L {
    static constexpr int BS = M2M_BS, MINB = 0;  // bounds on the block size only
    Coef<real> C;
    int l;
    int depth;
    const int *__restrict__ leaf_start;
    const real *__restrict__ loc_parent;
    real *__restrict__ loc_child;
    __device__ __forceinline__ void run(const int bid_, const int nblk_) const {
        constexpr int P3 = P * P * P, PP = P * P;
        extern __shared__ unsigned char smraw[];
        real *Lp = reinterpret_cast<real *>(smraw);  // [K][J][I]             p^3
        real *A = Lp + P3;                           // [hz][k][J][I]       2 p^3
        real *B = A + 2 * P3;                        // [hz][hy][k][j][I]   4 p^3
        real *Gs = B + 4 * P3;                       // [h][J][i]           2 p^2
        __shared__ unsigned occ_child;               // bit h: child h holds charges
        const int Hp = 1 << (l - 1);  // parents per axis (level l-1)
        const int pid = bid_;
        const int px = pid % Hp, py = (pid / Hp) % Hp, pz = pid / (Hp * Hp);
        const int64_t pkey = morton_encode(px, py, pz);
        if (!cell_occupied(leaf_start, depth, l - 1, pkey)) return;
        if (threadIdx.x < 32) {
            const bool o = threadIdx.x < 8 && cell_occupied(leaf_start, depth, l, pkey * 8 + threadIdx.x);
            const unsigned m = __ballot_sync(0xffffffffu, o);
            if (threadIdx.x == 0) occ_child = m;
        }
        const real *src = loc_parent + loc_cell(l - 1, px, py, pz) * P3;
        for (int e = threadIdx.x; e < 2 * PP; e += M2M_BS) Gs[e] = C.G[e / PP][e % PP];
        for (int o = threadIdx.x; o < P3; o += M2M_BS) Lp[o] = src[o];
        __syncthreads();
        for (int e = threadIdx.x; e < 2 * P3; e += M2M_BS) {
            const int hz = e / P3, o = e % P3, IJ = o % PP, k = o / PP;
            const real *g = Gs + hz * PP + k;
            real s = 0;
#pragma unroll
            for (int K = 0; K < P; K++) s += g[K * P] * Lp[K * PP + IJ];
            A[e] = s;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < 4 * P3; e += M2M_BS) {
            const int hh = e / P3, o = e % P3, I = o % P, j = (o / P) % P, k = o / PP;
            const int hz = hh >> 1, hy = hh & 1;
            const real *g = Gs + hy * PP + j;
            const real *a = A + hz * P3 + k * PP + I;
            real s = 0;
#pragma unroll
            for (int J = 0; J < P; J++) s += g[J * P] * a[J * P];
            B[e] = s;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < 8 * P3; e += M2M_BS) {
            const int h = e / P3, o = e % P3, i = o % P, row = o - i;
            const int hx = h & 1, hy = (h >> 1) & 1, hz = h >> 2;
            const real *g = Gs + hx * PP + i;
            const real *b = B + ((hz << 1) | hy) * P3 + row;
            real s = 0;
#pragma unroll
            for (int I = 0; I < P; I++) s += g[I * P] * b[I];
            const int cx = 2 * px + hx, cy = 2 * py + hy, cz = 2 * pz + hz;
            if (occ_child & (1u << h)) loc_child[loc_cell(l, cx, cy, cz) * P3 + o] += s;
        }
    }
};
template <typename real, int P>
__global__ void __launch_bounds__(KL2L<real, P>::BS) k_l2l(const __grid_constant__ KL2L<real, P> k) {
    k.run(blockIdx.x, gridDim.x);
}

template <typename real, int P>
constexpr size_t l2l_smem() {
    return sizeof(real) * (7 * P * P * P + 2 * P * P);
}

// ---------------------------------------------------------------------------
template <typename real>
void launch_upward(const Geom &g, const Coef<real> &C, const Ptrs<real> &P, const WsLayout &W,
                   cudaStream_t st, Tracer &tr) {
    const int p = g.p, p3 = g.p3, depth = g.depth;
    real *phi_leaf = P.phi + W.phi_level[depth];
    const int ncell = (int)W.ncell;
    tr.begin(FMM_STAGE_P2M, st);
    switch (p) {
#define WCASE(PP)                                                                                \
    case PP:                                                                                     \
        launch_k(tr, FMM_TAG(S_P2M, 0), k_p2m_warp<real, PP>,                                    \
                 KP2MWarp<real, PP>{C, depth, ncell, g.shift_free, P.leaf_start, P.s_pt, phi_leaf, \
                                    P.qlev + W.q_level[depth]},                                   \
                 (ncell + P2M_WARPS - 1) / P2M_WARPS, 32 * P2M_WARPS, 0, st);                     \
        break;
#define CASE(PP)                                                                                 \
    case PP:                                                                                     \
        launch_k(tr, FMM_TAG(S_P2M, 0), k_p2m<real, PP>,                                         \
                 KP2M<real, PP>{C, depth, P.leaf_start, P.s_pt, phi_leaf, P.qlev + W.q_level[depth]}, \
                 ncell, P2M_BS, 0, st);                                                           \
        break;
        WCASE(2) WCASE(3) WCASE(4) WCASE(5) WCASE(6) CASE(7) CASE(8)
#undef CASE
#undef WCASE
    }
    tr.count();
    tr.end();
    if (g.shift_free) {  // App. A.2: the box basis is additive over children
        if constexpr (std::is_same<real, double>::value) launch_sf_upward(g, P, W, st, tr);
        return;
    }
    tr.begin(FMM_STAGE_M2M, st);
    const int lmin = g.periodic ? 0 : 2;
    for (int l = depth; l >= 1; l--) {
        launch_halo<real>(p3, l, g.periodic, P.phi + W.phi_level[l], P.qlev + W.q_level[l], st, tr);
        tr.count();
        if (l - 1 >= lmin) {
            int nparent = 1 << (3 * (l - 1));
            switch (p) {
#define CASE(PP)                                                                                   \
    case PP:                                                                                       \
        launch_k(tr, FMM_TAG(S_M2M, l), k_m2m<real, PP>,                                          \
                 KM2M<real, PP>{C, l, P.phi + W.phi_level[l], P.phi + W.phi_level[l - 1],          \
                                P.qlev + W.q_level[l], P.qlev + W.q_level[l - 1], depth, P.leaf_start}, \
                 nparent, M2M_BS, m2m_smem<real, PP>(), st);                                      \
        break;
                CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8)
#undef CASE
            }
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
    const size_t sm_m2l = sizeof(real) * (M2L_T * M2L_PS + M2L_T * M2L_T + 2 * M2L_T);
    // 1. every level's own interaction-list contributions (they only need Phi),
    //    for every kernel component c (its own L block, forms scaled by
    //    2^(l spow)): L_0 = lattice term (periodic), L_l = sum over the
    //    interaction list
    const int lstart = g.periodic ? 1 : 2;
    if (g.periodic) {
        tr.begin(FMM_STAGE_M2L, st);
        for (int c = 0; c < T.ncomp; c++) {
            launch_k(tr, FMM_TAG(S_LATTICE, c), k_lattice<real>,
                     KLattice<real>{p3, T.Klt[c], T.Klbar[c], P.phi + W.phi_level[0], P.qlev + W.q_level[0],
                                    P.loc + c * W.loc_comp + W.loc_level[0]},
                     1, 256, 0, st);
            tr.count();
        }
        tr.end();
    }
    if (g.shift_free) {  // App. A.2: precomputed forms, identity downward pass
        if constexpr (std::is_same<real, double>::value)
            launch_sf_downward(g, P, W, T.sf_tab, T.sf_base, T.sf_H, T.sf_hoff, st, tr);
        return FMM_OK;
    }
    int lsimt_end = depth;
    if (T.tc_lmin > 0 && depth >= T.tc_lmin) lsimt_end = T.tc_lmin - 1;
    // the SIMT levels run on the coarse stream, beside the tensor-core levels
    if (!tr.rec) {
        cudaEventRecord(S.fork, st);
        cudaStreamWaitEvent(S.coarse, S.fork, 0);
    }
    for (int c = 0; c < T.ncomp; c++) {
        real *loc_c = P.loc + c * W.loc_comp;
        const int spow = c == 0 ? g.power : g.power + 1;  // 1/r^k: 2^(lk); its force: 2^(l(k+1))
        for (int l = lstart; l <= lsimt_end; l++) {
            const int H = 1 << (l - 1);
            const int Tt = H < 4 ? H : 4;
            const int ntiles = (H / Tt) * (H / Tt) * (H / Tt);
            const int G = m2l_groups(l, p3);
            real *dst = G > 1 ? P.m2l_part : loc_c + W.loc_level[l];
            tr.begin(FMM_STAGE_M2L, S.coarse);
            launch_k(tr, FMM_TAG(S_M2L_SIMT, 4 * l + c), k_m2l_simt<real>,
                     KM2LSimt<real>{p, l, P.phi + W.phi_level[l], P.qlev + W.q_level[l], dst, T.KtT[c], T.Kbar[c],
                                    G, spow, ntiles, P.leaf_start, depth},
                     ntiles * 8 * achunks * G, M2L_BS, sm_m2l, S.coarse);
            tr.count();
            if (G > 1) {
                const int64_t n = ((int64_t)1 << (3 * l)) * p3;
                int nb = (int)((n + 255) / 256);
                if (nb > 152 * 16) nb = 152 * 16;
                launch_k(tr, FMM_TAG(S_M2L_REDUCE, 4 * l + c), k_m2l_reduce<real>,
                         KM2LReduce<real>{G, n, P.m2l_part, loc_c + W.loc_level[l]}, nb, 256, 0, S.coarse);
                tr.count();
            }
            tr.end();
        }
    }
    if (!tr.rec) cudaEventRecord(S.coarse_done, S.coarse);
    if constexpr (std::is_same<real, float>::value) {
        if (T.tc_lmin > 0 && depth >= T.tc_lmin) {
            for (int c = 0; c < T.ncomp; c++) {
                int rc = launch_m2l_tc(g, P, W, T.tc_khi_map[c], T.tc_klo_map[c], T.tc_kbar[c], T.tc_lmin,
                                       T.tc_mode, T.tc_inject, P.loc + c * W.loc_comp,
                                       c == 0 ? g.power : g.power + 1,
                                       c == 0, c, st, tr);
                if (rc) return rc;
            }
        }
    }
    if (!tr.rec) cudaStreamWaitEvent(st, S.coarse_done, 0);
    // 2. downward: Psi_child = Psi_parent o shift, added level by level (the
    //    shift acts on functionals whatever their kernel)
    for (int c = 0; c < T.ncomp; c++) {
        real *loc_c = P.loc + c * W.loc_comp;
        for (int l = g.periodic ? 1 : 3; l <= depth; l++) {
            int nparent = 1 << (3 * (l - 1));
            tr.begin(FMM_STAGE_L2L, st);
            switch (p) {
#define CASE(PP)                                                                                   \
    case PP:                                                                                       \
        launch_k(tr, FMM_TAG(S_L2L, 4 * l + c), k_l2l<real, PP>,                                  \
                 KL2L<real, PP>{C, l, depth, P.leaf_start, loc_c + W.loc_level[l - 1], loc_c + W.loc_level[l]}, \
                 nparent, M2M_BS, l2l_smem<real, PP>(), st);                                      \
        break;
                CASE(2) CASE(3) CASE(4) CASE(5) CASE(6) CASE(7) CASE(8)
#undef CASE
            }
            tr.count();
            tr.end();
        }
    }
    return FMM_OK;
}

void far_set_attributes() {
    const int sm_simt_d = (int)(sizeof(double) * (M2L_T * M2L_PS + M2L_T * M2L_T + 2 * M2L_T));
    cudaFuncSetAttribute(k_m2l_simt<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm_simt_d);
    kb_set_smem<KM2LSimt<double>>(sm_simt_d);
#define ATTR(real, PP)                                                                             \
    cudaFuncSetAttribute(k_m2m<real, PP>, cudaFuncAttributeMaxDynamicSharedMemorySize,           \
                         (int)m2m_smem<real, PP>());                                              \
    cudaFuncSetAttribute(k_l2l<real, PP>, cudaFuncAttributeMaxDynamicSharedMemorySize,           \
                         (int)l2l_smem<real, PP>());                                              \
    kb_set_smem<KM2M<real, PP>>(m2m_smem<real, PP>());                                           \
    kb_set_smem<KL2L<real, PP>>(l2l_smem<real, PP>());
    ATTR(float, 2) ATTR(float, 3) ATTR(float, 4) ATTR(float, 5) ATTR(float, 6) ATTR(float, 7)
    ATTR(float, 8) ATTR(double, 2) ATTR(double, 3) ATTR(double, 4) ATTR(double, 5)
    ATTR(double, 6) ATTR(double, 7) ATTR(double, 8)
#undef ATTR
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

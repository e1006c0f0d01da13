// App. A.2: bilinear forms without shifts (double-precision plans).
//
// Every cell's grid charges are taken with respect to the box S:
// Phi^S_C = shift_{C->S}(Phi_C), which is also the replacement of C's charges
// directly with respect to S.  The box basis is additive over children, so
// the upward pass is a sum; the functional of a cell, taken with respect to S
// as well, passes unchanged to its children (the downward pass is the
// identity), and the interaction lists apply
//     BB_{C~,o} = shift_{S->C~}^T  K_o  shift_{S->C},   C = C~ + o,
// computed once per plan.  shift_{S->C} is the inverse of shift_{C->S}; along
// one axis its entry (i, b) is the cell's basis function i at the box node b
// in cell coordinates, g_i(2^l a_b - c), since the box basis is exact on
// polynomials of degree < p.  It extrapolates over 2^l cells, hence FP64.
//
// Every form of a target C~ has the same left factor shift_{S->C~}^T, so a
// form is stored as its right part A_{C~,o} = K_o shift_{S->C} (p^3 x p^3 per
// cell and offset) and the left factor is applied once per target, after the
// sum over the interaction list.  Stored as the full product, the rounding of
// each entry (|BB| ~ 1e15 at level 3, order 4) is read back through the box
// weights at full size: 5e-6 relative in the far field there, against 3e-9
// for the factored sum, whose rounding inside the cell basis the left factor
// and the box weights cancel exactly (g^S(x) . shift_{S->C~}^T y = g^C~(x) . y).
#include <cmath>
#include <vector>

#include "fmm_internal.cuh"

namespace fmm {

#define SF_TBS 256  // threads of the table kernel
#define SF_BS 512   // threads of the contraction kernel
#define SF_NOFF 189

// cell (cx, cy, cz) of level l >= 1 from its index in the L layout
__device__ inline void sf_loc_decode(int l, int64_t cl, int &cx, int &cy, int &cz) {
    const int64_t H = (int64_t)1 << (l - 1);
    const int hx = (int)(cl % H), hy = (int)((cl / H) % H), hz = (int)((cl / (H * H)) % H);
    const int par = (int)(cl / (H * H * H));
    cx = 2 * hx + (par & 1);
    cy = 2 * hy + ((par >> 1) & 1);
    cz = 2 * hz + ((par >> 2) & 1);
}

// offset oi (0..188) of the interaction list of a target of parity (bx, by,
// bz): the children of the parent's 27-cell neighbourhood, [-2-b, 3-b] per
// axis, without the 27 cells adjacent to the target; x fastest
__device__ inline void sf_offset(int oi, int bx, int by, int bz, int &ox, int &oy, int &oz) {
    int k = -1;
    ox = oy = oz = 0;
    for (int z = -2 - bz; z <= 3 - bz; z++)
        for (int y = -2 - by; y <= 3 - by; y++)
            for (int x = -2 - bx; x <= 3 - bx; x++) {
                if (x >= -1 && x <= 1 && y >= -1 && y <= 1 && z >= -1 && z <= 1) continue;
                if (++k == oi) {
                    ox = x;
                    oy = y;
                    oz = z;
                    return;
                }
            }
}

// source cell of offset (ox, oy, oz) from target (cx, cy, cz): wrapped in the
// periodic form, false when outside the box in the open form
__device__ inline bool sf_source(int S, int periodic, int cx, int cy, int cz, int ox, int oy, int oz,
                                 int &sx, int &sy, int &sz) {
    sx = cx + ox;
    sy = cy + oy;
    sz = cz + oz;
    if (periodic) {
        sx = (sx % S + S) % S;
        sy = (sy % S + S) % S;
        sz = (sz % S + S) % S;
        return true;
    }
    return sx >= 0 && sy >= 0 && sz >= 0 && sx < S && sy < S && sz < S;
}

// ---------------------------------------------------------------------------
// The right parts of one level: one CTA per (target cell, offset).  M = K_o
// (unit cells, [target cell node][source cell node]) in shared memory, then
// three in-place passes of p-point transforms, M <- M shift_{S->C} along the
// source axes.  Written transposed and scaled to unit-box units:
// tab[n][m] = 2^l A[m][n] (n a box node of the source, m a node of the target
// cell).  H: [c][i][b] = shift_{S->C} along one axis for coordinate c of
// level l.  Pairs whose source lies outside the open box are never read: not
// written.
// ---------------------------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(SF_TBS) k_sf_table(Coef<double> C, int l, int periodic,
                                                     const double *__restrict__ H,
                                                     double *__restrict__ tab_l) {
    constexpr int P3 = P * P * P, PP = P * P;
    constexpr int64_t P6 = (int64_t)P3 * P3;
    extern __shared__ double sm[];
    double *M = sm;       // [P3][P3]
    double *Hs = sm + P6;  // [3][i][b]: source x, y, z
    const int64_t pair = blockIdx.x;
    const int64_t cl = pair / SF_NOFF;
    const int oi = (int)(pair % SF_NOFF);
    const int S = 1 << l;
    int cx, cy, cz, ox, oy, oz, sx, sy, sz;
    sf_loc_decode(l, cl, cx, cy, cz);
    sf_offset(oi, cx & 1, cy & 1, cz & 1, ox, oy, oz);
    if (!sf_source(S, periodic, cx, cy, cz, ox, oy, oz, sx, sy, sz)) return;  // uniform over the CTA
    const int cc[3] = {sx, sy, sz};
    for (int e = threadIdx.x; e < 3 * PP; e += SF_TBS) Hs[e] = H[(int64_t)cc[e / PP] * PP + e % PP];
    for (int64_t e = threadIdx.x; e < P6; e += SF_TBS) {
        const int a = (int)(e / P3), b = (int)(e % P3);
        const double dx = C.tau[a % P] - (ox + C.tau[b % P]);
        const double dy = C.tau[(a / P) % P] - (oy + C.tau[(b / P) % P]);
        const double dz = C.tau[a / PP] - (oz + C.tau[b / PP]);
        M[e] = 1.0 / sqrt(dx * dx + dy * dy + dz * dz);
    }
    __syncthreads();
    int64_t stride = 1;  // digit `pass` of the 6-digit (base p) index of M
    for (int pass = 0; pass < 3; pass++, stride *= P) {
        const double *Hm = Hs + pass * PP;
        for (int64_t L = threadIdx.x; L < P6 / P; L += SF_TBS) {
            const int64_t base = (L / stride) * stride * P + L % stride;
            double v[P];
#pragma unroll
            for (int i = 0; i < P; i++) v[i] = M[base + i * stride];
#pragma unroll
            for (int b = 0; b < P; b++) {
                double s = 0.0;
#pragma unroll
                for (int i = 0; i < P; i++) s += v[i] * Hm[i * P + b];
                M[base + b * stride] = s;
            }
        }
        __syncthreads();
    }
    double *out = tab_l + pair * P6;
    const double sc = (double)S;
    for (int64_t e = threadIdx.x; e < P6; e += SF_TBS) {
        const int n = (int)(e / P3), m = (int)(e % P3);
        out[e] = sc * M[(int64_t)m * P3 + n];
    }
}

template <int P>
constexpr size_t sf_table_smem() {
    return sizeof(double) * ((size_t)P * P * P * P * P * P + 3 * P * P);
}

// ---------------------------------------------------------------------------
// Upward pass: Phi^S_parent = sum of the eight children (x fastest), and the
// cells' total charges likewise.  Children of level l, parents of l - 1.
// ---------------------------------------------------------------------------
__global__ void k_sf_up(int l, int p3, const double *__restrict__ phi_c, double *__restrict__ phi_p,
                        const double *__restrict__ q_c, double *__restrict__ q_p) {
    const int Sp = 1 << (l - 1);
    const int64_t items = (int64_t)Sp * Sp * Sp * (p3 + 1);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < items;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t pc = e / (p3 + 1);
        const int o = (int)(e % (p3 + 1));
        const int px = (int)(pc % Sp), py = (int)((pc / Sp) % Sp), pz = (int)(pc / ((int64_t)Sp * Sp));
        double s = 0.0;
        for (int h = 0; h < 8; h++) {
            const int64_t c = phi_cell(l, 2 * px + (h & 1), 2 * py + ((h >> 1) & 1), 2 * pz + (h >> 2));
            s += o < p3 ? phi_c[c * p3 + o] : q_c[c];
        }
        const int64_t pcell = phi_cell(l - 1, px, py, pz);
        if (o < p3) phi_p[pcell * p3 + o] = s;
        else q_p[pcell] = s;
    }
}

// ---------------------------------------------------------------------------
// Interaction lists of level l:
//     L^S_C~ = L^S_parent + shift_{S->C~}^T sum_o A_{C~,o} Phi^S_{C~+o}.
// One CTA per target cell, 16 warps; warp w takes the offsets w, w + 16, ...
// and lane t the target nodes t, t + 32, ... (its table columns are
// contiguous over the warp).  The source vector sits in the lanes' registers
// and is broadcast by shuffles; even and odd source nodes go to two
// accumulators.  The warps' sums are added in warp order, then the left
// factor is applied by three in-place passes of p-point transforms.
// ---------------------------------------------------------------------------
template <int P>
__global__ void __launch_bounds__(SF_BS) k_sf_m2l(int l, int periodic, int add_parent,
                                                  const double *__restrict__ phi_l,
                                                  const double *__restrict__ tab_l,
                                                  const double *__restrict__ H,
                                                  const double *__restrict__ loc_parent,
                                                  double *__restrict__ loc_l) {
    constexpr int P3 = P * P * P, PP = P * P;
    constexpr int64_t P6 = (int64_t)P3 * P3;
    constexpr int MR = (P3 + 31) / 32;  // target nodes per lane
    constexpr int NW = SF_BS / 32;
    __shared__ int64_t src[SF_NOFF];
    __shared__ double part[NW][MR * 32];
    __shared__ double y[P3];
    __shared__ double Ht[3][PP];
    const int64_t cl = blockIdx.x;
    const int S = 1 << l;
    int cx, cy, cz;
    sf_loc_decode(l, cl, cx, cy, cz);
    for (int oi = threadIdx.x; oi < SF_NOFF; oi += SF_BS) {
        int ox, oy, oz, sx, sy, sz;
        sf_offset(oi, cx & 1, cy & 1, cz & 1, ox, oy, oz);
        src[oi] = sf_source(S, periodic, cx, cy, cz, ox, oy, oz, sx, sy, sz) ? phi_cell(l, sx, sy, sz) : -1;
    }
    for (int e = threadIdx.x; e < 3 * PP; e += SF_BS) {
        const int c = e < PP ? cx : e < 2 * PP ? cy : cz;
        Ht[e / PP][e % PP] = H[(int64_t)c * PP + e % PP];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double a0[MR], a1[MR];
#pragma unroll
    for (int k = 0; k < MR; k++) a0[k] = a1[k] = 0.0;
    for (int oi = warp; oi < SF_NOFF; oi += NW) {
        const int64_t sc = src[oi];  // uniform over the warp
        if (sc < 0) continue;
        const double *B = tab_l + (cl * SF_NOFF + oi) * P6 + lane;
        const double *ph = phi_l + sc * P3;
        double f[MR];
#pragma unroll
        for (int k = 0; k < MR; k++) f[k] = (lane + 32 * k < P3) ? ph[lane + 32 * k] : 0.0;
#pragma unroll
        for (int n = 0; n < P3; n++) {
            const double v = __shfl_sync(0xffffffffu, f[n >> 5], n & 31);
#pragma unroll
            for (int k = 0; k < MR; k++) {
                if (32 * k + 32 <= P3 || lane + 32 * k < P3) {
                    const double b = B[(int64_t)n * P3 + 32 * k];
                    if (n & 1) a1[k] += b * v;
                    else a0[k] += b * v;
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < MR; k++) part[warp][lane + 32 * k] = a0[k] + a1[k];
    __syncthreads();
    if (threadIdx.x < P3) {
        double t = part[0][threadIdx.x];
#pragma unroll
        for (int w = 1; w < NW; w++) t += part[w][threadIdx.x];
        y[threadIdx.x] = t;
    }
    __syncthreads();
    // y <- shift_{S->C~}^T y along x, y, z (node index (k*p + j)*p + i)
    int stride = 1;
    for (int ax = 0; ax < 3; ax++, stride *= P) {
        if (threadIdx.x < PP) {
            const int L = threadIdx.x;
            const int base = (L / stride) * stride * P + L % stride;
            double v[P];
#pragma unroll
            for (int i = 0; i < P; i++) v[i] = y[base + i * stride];
#pragma unroll
            for (int b = 0; b < P; b++) {
                double s = 0.0;
#pragma unroll
                for (int i = 0; i < P; i++) s += v[i] * Ht[ax][i * P + b];
                y[base + b * stride] = s;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x < P3) {
        const double s = add_parent ? loc_parent[loc_cell(l - 1, cx >> 1, cy >> 1, cz >> 1) * P3 + threadIdx.x] : 0.0;
        loc_l[cl * P3 + threadIdx.x] = s + y[threadIdx.x];
    }
}

// ---------------------------------------------------------------------------
size_t sf_table_bytes(int p, int depth, int periodic, int64_t *base) {
    const int64_t p6 = (int64_t)p * p * p * p * p * p;
    int64_t pairs = 0;
    for (int l = 0; l <= depth + 1; l++) base[l] = 0;
    for (int l = periodic ? 1 : 2; l <= depth; l++) {
        base[l] = pairs;
        pairs += ((int64_t)1 << (3 * l)) * SF_NOFF;
    }
    return (size_t)pairs * p6 * sizeof(double);
}

int sf_build(int p, int depth, int periodic, const Coef<double> &C, void **tab, int64_t *base,
             void **hmat, int64_t *hoff_out) {
    const size_t bytes = sf_table_bytes(p, depth, periodic, base);
    const int pp = p * p;
    // per-axis shift_{S->C}: [l][c][i][b] = g_i(2^l a_b - c), levels 1..depth
    std::vector<double> h;
    std::vector<int64_t> hoff(depth + 2, 0);
    for (int l = 1; l <= depth; l++) {
        hoff[l] = (int64_t)h.size();
        const int S = 1 << l;
        for (int c = 0; c < S; c++)
            for (int i = 0; i < p; i++)
                for (int b = 0; b < p; b++) {
                    const double x = S * ((double)b / (p - 1)) - c;
                    double v = 1.0;
                    for (int k = 0; k < p; k++)
                        if (k != i) v *= (x - (double)k / (p - 1)) / ((double)(i - k) / (p - 1));
                    h.push_back(v);
                }
    }
    double *dH = nullptr, *dT = nullptr;
    if (cudaMalloc(&dH, h.size() * sizeof(double)) != cudaSuccess) return FMM_ERR_OOM;
    if (cudaMalloc(&dT, bytes) != cudaSuccess) {
        cudaFree(dH);
        cudaGetLastError();
        return FMM_ERR_OOM;
    }
    int rc = FMM_OK;
    if (cudaMemcpy(dH, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
        rc = FMM_ERR_CUDA;
    const int64_t p6 = (int64_t)pp * pp * pp;
    for (int l = periodic ? 1 : 2; l <= depth && rc == FMM_OK; l++) {
        const int64_t pairs = ((int64_t)1 << (3 * l)) * SF_NOFF;
        double *out = dT + base[l] * p6;
        switch (p) {
#define CASE(PP)                                                                                   \
    case PP:                                                                                       \
        cudaFuncSetAttribute(k_sf_table<PP>, cudaFuncAttributeMaxDynamicSharedMemorySize,          \
                             (int)sf_table_smem<PP>());                                            \
        k_sf_table<PP><<<(unsigned)pairs, SF_TBS, sf_table_smem<PP>()>>>(C, l, periodic,           \
                                                                         dH + hoff[l], out);        \
        break;
            CASE(2) CASE(3) CASE(4) CASE(5)
#undef CASE
        default: rc = FMM_ERR_UNSUPPORTED;
        }
        if (cudaGetLastError() != cudaSuccess) rc = FMM_ERR_CUDA;
    }
    if (rc == FMM_OK && cudaDeviceSynchronize() != cudaSuccess) rc = FMM_ERR_CUDA;
    if (rc != FMM_OK) {
        cudaFree(dH);
        cudaFree(dT);
        return rc;
    }
    *tab = dT;
    *hmat = dH;
    for (int l = 0; l <= depth + 1; l++) hoff_out[l] = l <= depth ? hoff[l] : 0;
    return FMM_OK;
}

void launch_sf_upward(const Geom &g, const Ptrs<double> &P, const WsLayout &W, cudaStream_t st,
                      Tracer &tr) {
    const int lmin = g.periodic ? 0 : 2;
    tr.begin(FMM_STAGE_M2M, st);
    for (int l = g.depth; l > lmin; l--) {
        const int64_t items = ((int64_t)1 << (3 * (l - 1))) * (g.p3 + 1);
        int nb = (int)((items + 255) / 256);
        if (nb > 152 * 16) nb = 152 * 16;
        k_sf_up<<<nb, 256, 0, st>>>(l, g.p3, P.phi + W.phi_level[l], P.phi + W.phi_level[l - 1],
                                    P.qlev + W.q_level[l], P.qlev + W.q_level[l - 1]);
        tr.count();
    }
    tr.end();
}

void launch_sf_downward(const Geom &g, const Ptrs<double> &P, const WsLayout &W, const double *tab,
                        const int64_t *base, const double *hmat, const int64_t *hoff,
                        cudaStream_t st, Tracer &tr) {
    const int64_t p6 = (int64_t)g.p3 * g.p3;
    for (int l = g.periodic ? 1 : 2; l <= g.depth; l++) {
        const int add_parent = g.periodic ? 1 : (l >= 3);
        const double *phi_l = P.phi + W.phi_level[l], *tab_l = tab + base[l] * p6;
        const double *loc_p = P.loc + W.loc_level[l - 1];
        double *loc_l = P.loc + W.loc_level[l];
        const unsigned ncell = 1u << (3 * l);
        tr.begin(FMM_STAGE_M2L, st);
        switch (g.p) {
#define CASE(PP)                                                                                    \
    case PP:                                                                                        \
        k_sf_m2l<PP><<<ncell, SF_BS, 0, st>>>(l, g.periodic, add_parent, phi_l, tab_l,            \
                                              hmat + hoff[l], loc_p, loc_l);                         \
        break;
            CASE(2) CASE(3) CASE(4) CASE(5)
#undef CASE
        }
        tr.count();
        tr.end();
    }
}

}  // namespace fmm

// Internal declarations of the GB300 replacement-FMM library (not part of the C ABI).
//
// Data layout in device memory (all indices int32 unless noted):
//   charges after binning/split, sorted by finest cell (Morton order):
//     s_pt[slot]     real4 (t_x, t_y, t_z, q_eff): t in finest-cell units, [0,1]
//     s_origin[slot] particle the charge came from
//   grid charges Phi of level l >= 1: 8 parity blocks of (H+2)^3 coarse cells
//     (H = 2^(l-1); one halo cell per side, zero in the open form, the periodic
//     image in the periodic form), each cell a contiguous p^3 vector with node
//     (i,j,k) at (k*p + j)*p + i.  Level 0 is a single cell.
//   functionals L of level l >= 1: 8 parity blocks of H^3 cells (no halo).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/fmm_gb300.h"

#define FMM_MAXP 8
#define FMM_MAXDEPTH 8

namespace fmm {

// Coefficients of the p-division points of the unit segment (§2.1.2) and of the
// child->parent shift (eq. trans), in the plan's real type.  Passed by value.
template <typename real>
struct Coef {
    real tau[FMM_MAXP];                    // nodes i/(p-1)
    real cinv[FMM_MAXP];                   // 1 / prod_{k != i} (tau_i - tau_k)
    real G[2][FMM_MAXP * FMM_MAXP];        // G_h[J*p + i] = g_J((h + tau_i)/2)
};

// Per-evaluation scalars.
struct Geom {
    int p, p3, depth, periodic, continuous, force_mode;
    int shift_free;   // App. A.2: grid charges and functionals with respect to the box
    int power;        // F(P, P~) = 1/r^power: 1 (Coulomb) or 2
    int S;            // 2^depth
    float x0[3];      // float32 box corner
    float Lf;         // float32 box edge
    float dtf, dthi;  // split half-width in finest-cell units and 1 - dtf (float32)
    double L;         // box edge (FP64) for output scaling
};

// Workspace header (first 256 bytes of the workspace).
struct WsHeader {
    int status;       // FMM_ERR_* bits from the device (see status codes below)
    int n_eff;        // charges after the split
    int n_coinc;      // coincident pairs skipped in the near field
    int valid;        // 0 until an evaluation completed
    long long tag;    // plan id and n of the last evaluation
    // first bounded wait that gave up: site (1 producer slot, 2 MMA region,
    // 3 MMA operands, 4 epilogue region), block, level, iteration
    int wait_site, wait_block, wait_level, wait_iter;
};

// device-side status bits
#define ST_OUT_OF_BOX 1
#define ST_NONFINITE 2
#define ST_SPLIT_OVERFLOW 4
#define ST_TIMEOUT 8
#define ST_STATE 16  // backward on a workspace whose last evaluation was another plan's or n's

// Workspace carving (byte offsets), computed on the host for (plan, n).
struct WsLayout {
    size_t hdr;
    size_t count, offset, axes;           // per particle (continuous form)
    size_t e_key, e_pt, e_wd, e_origin;   // per emitted charge (e_pt: results after the sort)
    size_t e_rank;                        // arrival rank of each emitted charge in its cell
    size_t leaf_count, leaf_start;
    size_t tmp, perm;
    size_t s_pt, s_origin, out_pt;
    size_t react;  // [13][cap] near-field reactions per forward direction (mutual near field)
    size_t phi, loc;                      // all levels (loc: ncomp blocks of loc_comp)
    size_t qlev;                          // total charge of every cell, padded Phi layout
    size_t phihi, philo;                  // TF32 split of Phi (tensor-core plans)
    size_t m2l_part;                      // per-offset-group partials of the SIMT contraction
    size_t occ;                           // occupied-cell lists of the contraction (tensor-core plans)
    size_t delta;                         // per emitted charge of a split particle: phi(s_k) - phi(r)
    size_t slist;                         // the split particles (count, then indices)
    size_t pord;                          // near-field launch order: class counts, fill, cells
    size_t scan_tmp, epart;
    size_t total;
    int64_t cap;                          // charge capacity
    int64_t ncell;                        // 8^depth
    int64_t phi_level[FMM_MAXDEPTH + 2];  // element offset of each level in Phi
    int64_t loc_level[FMM_MAXDEPTH + 2];  // element offset of each level in L
    int64_t loc_comp;                     // elements of one kernel component's L
    int64_t q_level[FMM_MAXDEPTH + 2];    // cell offset of each level in qlev
    int scan_blocks;
};

// ---- index helpers -----------------------------------------------------------
__host__ __device__ inline uint32_t morton_encode(uint32_t x, uint32_t y, uint32_t z) {
    uint32_t k = 0;
#pragma unroll
    for (int b = 0; b < 10; b++) {
        k |= ((x >> b) & 1u) << (3 * b);
        k |= ((y >> b) & 1u) << (3 * b + 1);
        k |= ((z >> b) & 1u) << (3 * b + 2);
    }
    return k;
}
__host__ __device__ inline void morton_decode(uint32_t k, int &x, int &y, int &z) {
    x = y = z = 0;
#pragma unroll
    for (int b = 0; b < 10; b++) {
        x |= (int)((k >> (3 * b)) & 1u) << b;
        y |= (int)((k >> (3 * b + 1)) & 1u) << b;
        z |= (int)((k >> (3 * b + 2)) & 1u) << b;
    }
}
// cell (cx,cy,cz) of level l >= 1 in the padded Phi layout
__host__ __device__ inline int64_t phi_cell(int l, int cx, int cy, int cz) {
    if (l == 0) return 0;
    int64_t H = (int64_t)1 << (l - 1), P = H + 2;
    int par = (cx & 1) | ((cy & 1) << 1) | ((cz & 1) << 2);
    return ((par * P + (cz >> 1) + 1) * P + (cy >> 1) + 1) * P + (cx >> 1) + 1;
}
__host__ __device__ inline int64_t phi_level_cells(int l) {
    if (l == 0) return 1;
    int64_t P = ((int64_t)1 << (l - 1)) + 2;
    return 8 * P * P * P;
}
// Tensor-core operand layout of the grid charges (split hi / lo copies): the
// padded parity-major layout with at least 10 cells per axis, so that every
// 8 x 4 x 4 box the contraction loads (starting at coarse coordinate 0..2)
// lies inside the grid; cells beyond the padded layout hold zeros.
__host__ __device__ inline int64_t tc_level_extent(int l) {
    int64_t P = ((int64_t)1 << (l - 1)) + 2;
    return P < 10 ? 10 : P;
}
__host__ __device__ inline int64_t tc_level_cells(int l) {
    if (l == 0) return 1;
    int64_t Pt = tc_level_extent(l);
    return 8 * Pt * Pt * Pt;
}
__host__ __device__ inline int64_t tc_level_first(int l) {  // cells before level l
    int64_t c = 0;
    for (int k = 0; k < l; k++) c += tc_level_cells(k);
    return c;
}

// cell of level l >= 1 in the unpadded L layout
__host__ __device__ inline int64_t loc_cell(int l, int cx, int cy, int cz) {
    if (l == 0) return 0;
    int64_t H = (int64_t)1 << (l - 1);
    int par = (cx & 1) | ((cy & 1) << 1) | ((cz & 1) << 2);
    return ((par * H + (cz >> 1)) * H + (cy >> 1)) * H + (cx >> 1);
}
__host__ __device__ inline int64_t loc_level_cells(int l) { return (int64_t)1 << (3 * l); }

// A cell of level l with Morton key k holds charges iff its finest cells
// [k 8^(depth-l), (k+1) 8^(depth-l)) hold any: their sorted ranges do not
// all start at the same slot.
__device__ __forceinline__ bool cell_occupied(const int *leaf_start, int depth, int l, int64_t key) {
    const int sh = 3 * (depth - l);
    return leaf_start[(key + 1) << sh] > leaf_start[key << sh];
}

// Occupied-cell lists of the tensor-core contraction: one segment per (level
// l >= lmin, target parity), s = 8 (l - lmin) + parity, holding the occupied
// cells of that parity in coarse Morton order; the lists are built in blocks
// of OCC_BLOCK coarse cells.  Ints in the workspace region `occ`:
//   [0, nblk)                     occupied cells per block (then their prefix)
//   [nblk, nblk + nseg)           occupied cells per segment
//   [.., + nseg + 1)              prefix of the segments' 128-row tiles
//   [occ_list_offset, ..)         the lists, segment s from the number of
//                                 cells of the segments before it
#define OCC_BLOCK 1024
__host__ __device__ inline int occ_nseg(int depth, int lmin) { return 8 * (depth - lmin + 1); }
__host__ __device__ inline int64_t occ_seg_cells(int lmin, int s) { return (int64_t)1 << (3 * (lmin + s / 8 - 1)); }
__host__ __device__ inline int64_t occ_seg_first(int lmin, int s) {  // first list entry of segment s
    int64_t b = 0;
    for (int k = 0; k < s; k++) b += occ_seg_cells(lmin, k);
    return b;
}
__host__ __device__ inline int occ_nblk(int depth, int lmin) {
    int nb = 0;
    for (int s = 0; s < occ_nseg(depth, lmin); s++) nb += (int)((occ_seg_cells(lmin, s) + OCC_BLOCK - 1) / OCC_BLOCK);
    return nb;
}
__host__ __device__ inline int64_t occ_list_offset(int depth, int lmin) {
    return ((int64_t)occ_nblk(depth, lmin) + 2 * occ_nseg(depth, lmin) + 1 + 63) / 64 * 64;
}
// A segment takes box tiles (each offset's A operand one TMA box of 8 x 4 x 4
// coarse cells, empty cells included) when it has fewer than 8 coarse cells
// per axis or when the share of its cells that hold charges reaches the
// threshold of the tile width N (p^3 padded): the gathered tiles of narrow
// shapes keep fewer copies in flight per MMA, so they pay off only on sparser
// segments (measured: N = 224 gathers as fast as boxes, N = 128 at ~2/3 of
// their rate, N <= 64 at ~2/5).
__host__ __device__ inline bool occ_box_segment(int H, int64_t count, int N) {
    const int pct = N >= 224 ? 95 : (N >= 128 ? 70 : 40);
    return H < 8 || count * 100 >= (int64_t)pct * H * H * H;
}
__host__ __device__ inline int occ_seg_tiles(int H, int64_t count, int N) {
    if (count == 0) return 0;
    if (H < 8) return 1;
    return occ_box_segment(H, count, N) ? (int)((int64_t)H * H * H / 128) : (int)((count + 127) / 128);
}
__host__ __device__ inline int64_t occ_ints(int depth, int lmin) {
    return occ_list_offset(depth, lmin) + occ_seg_first(lmin, occ_nseg(depth, lmin));
}

template <typename real> struct Vec4;
template <> struct Vec4<float> { typedef float4 T; };
template <> struct Vec4<double> { typedef double4 T; };

struct LaunchRec;  // launch.cuh

// Stage tracer: counts kernel launches and, when on, brackets each stage's
// kernels with CUDA events on the stream (FMM_STAGE_* ids).  rec: the
// launches are recorded there instead of issued (batched evaluations merge
// them across systems; nothing but launches of functor kernels may be issued
// then: no memset, copy or event).
struct Tracer {
    std::vector<LaunchRec> *rec = nullptr;
    cudaStream_t near = nullptr;  // while recording: the near-field stream
    // while recording a batch whose small levels run as cross-system tiles:
    // the first level of a system's own tensor-core contraction
    int tc_lbig = 0;
    bool on = false;
    cudaStream_t st = 0;
    int launches = 0;
    cudaEvent_t *ev = nullptr;
    int cap = 0, n = 0;
    int stage[512];
    cudaStream_t cur = 0;
    // stage events on `stream` (default: the call's stream)
    void begin(int s, cudaStream_t stream = nullptr) {
        cur = stream ? stream : st;
        if (on && n + 2 <= cap) {
            stage[n / 2] = s;
            cudaEventRecord(ev[n++], cur);
        }
    }
    void end() {
        if (on && (n & 1)) cudaEventRecord(ev[n++], cur);
    }
    void count(int k = 1) { launches += k; }
};

// ---- kernels launch wrappers (defined in the .cu files) -------------------
template <typename real>
struct Ptrs {
    WsHeader *hdr;
    int *count, *offset;
    unsigned char *axes;
    uint32_t *e_key;
    typename Vec4<real>::T *e_pt, *e_wd;
    int *e_origin, *e_rank;
    int *leaf_count, *leaf_start;
    int *tmp, *perm;
    // per emitted charge, once the sort has consumed e_pt: (phi, F) of every
    // charge in unit-box units, written by the far field at the charges
    typename Vec4<real>::T *out_e;
    typename Vec4<real>::T *s_pt;
    int *s_origin;
    typename Vec4<real>::T *out_pt;
    typename Vec4<real>::T *react;
    real *phi, *loc;
    real *qlev;
    real *phihi, *philo;
    real *m2l_part;
    int *occ;
    float *delta;  // single-precision plans of the continuous form (adjoint split forces)
    int *slist;
    int *pord;
    int *scan_tmp;
    double *epart;
};

// Bilinear-form tables on the device.  K_o = Kbar_o[a] + Kt_o[a,b] with
// Kbar_o[a] = mean_b K_o[a,b]: the contraction sum_b K_o[a,b] Phi[b] is evaluated
// as sum_b Kt_o[a,b] Phi[b] + Kbar_o[a] Q with Q = sum_b Phi[b] the cell's total
// charge (replacement conserves charge), which removes the cancellation of the
// nearly constant kernel against grid charges of both signs.
// Component c of every table: c = 0 the potential kernel 1/r, c = 1..3 the
// force kernel r/|r|^3 (FMM_FORCE_KERNEL plans, ncomp = 4), whose forms scale
// by 4^l instead of 2^l at level l.
template <typename real>
struct DevTables {
    int ncomp;
    const real *KtT[4];    // [343][b][a] = Kt_o[a,b] (transposed, SIMT contraction)
    const real *Kbar[4];   // [343][a]
    const real *Klt[4];    // [a][b] lattice kernel minus its row mean (periodic form)
    const real *Klbar[4];  // [a]
    // tensor-core contraction (TF32X3 / TF32X1 / BF16X3 plans): levels >= tc_lmin, 0 = none
    int tc_lmin;
    int tc_mode;                          // FMM_TC_*
    int tc_inject;                        // FMM_INJECT_* test hook for this evaluation
    const void *tc_khi_map[4], *tc_klo_map[4];  // CUtensorMap of the split unit-cell kernels
    const float *tc_kbar[4];                    // [343][p3 padded to 32] row means
    // App. A.2 forms (shift-free plans), FP64: right parts K_o shift_{S->C},
    // [level pairs from sf_base[l]][n][m]; per-axis shift_{S->C} of every level
    // from sf_hoff[l], [c][i][b]
    const double *sf_tab;
    const int64_t *sf_base;
    const double *sf_H;
    const int64_t *sf_hoff;
};

// Offset groups of the SIMT contraction at level l: the 189 offsets of a
// target tile are split over G CTAs when a level has too few tiles to fill
// the GPU; each CTA writes a partial, summed afterwards in a fixed order.
__host__ __device__ inline int m2l_groups(int l, int p3) {
    int H = 1 << (l - 1), T = H < 4 ? H : 4;
    int ctas = (H / T) * (H / T) * (H / T) * 8 * ((p3 + 63) / 64);
    int G = (2 * 152 + ctas - 1) / ctas;
    return G < 1 ? 1 : (G > 27 ? 27 : G);
}

// tree / bookkeeping stage (kernels_tree.cu)
template <typename real>
void launch_bin_emit(const Geom &g, const Coef<real> &C, const Ptrs<real> &P, const WsLayout &W,
                     int n, const float *pos, const float *q, cudaStream_t st, Tracer &tr);
template <typename real>
void launch_sort(const Geom &g, const Ptrs<real> &P, const WsLayout &W, int n, cudaStream_t st,
                 Tracer &tr);
template <typename real>
void launch_unsplit(const Geom &g, const Ptrs<real> &P, const WsLayout &W, int n, const float *q,
                    real *potential, double *energy, real *forces, const double *grad_energy,
                    real *grad_q, bool backward, cudaStream_t st, Tracer &tr);
// single-precision plans, continuous form, adjoint forces: the potential
// differences between each split particle's charges (kernels_tree.cu)
void launch_split_delta(const Geom &g, const Coef<double> &Cd, const Ptrs<float> &P, const WsLayout &W, int n,
                        const float *pos, cudaStream_t st, Tracer &tr);
int launch_scan(const int *in, int *out, int m, int *tmp, cudaStream_t st, Tracer &tr);

// far field (kernels_far.cu)
template <typename real>
void launch_upward(const Geom &g, const Coef<real> &C, const Ptrs<real> &P, const WsLayout &W,
                   cudaStream_t st, Tracer &tr);
// Streams of one evaluation: the caller's stream, two plan-owned auxiliary
// streams and the events that fork work onto them and join it back.
struct Streams {
    cudaStream_t main, near, coarse;
    cudaEvent_t sorted, near_done, fork, coarse_done;
    cudaStream_t far;     // optional: the far-field chain's stream
    cudaEvent_t far_done;
};

template <typename real>
int launch_downward(const Geom &g, const Coef<real> &C, const Ptrs<real> &P, const WsLayout &W,
                    const DevTables<real> &T, const Streams &S, Tracer &tr);

// tensor-core contraction (m2l_tc.cu)
#define FMM_TC_TF32X3 0  // 3-pass split TF32
#define FMM_TC_TF32X1 1  // 1-pass TF32
#define FMM_TC_BF16X3 2  // 3-pass split BF16
// loc: the functionals to write (one kernel component); spow: forms scale by
// 2^(l spow) at level l; split: also split the grid charges into the operand
// copies (once per evaluation)
// one system of a batched evaluation's cross-system contraction tiles
struct TcXSys {
    const char *op_hi, *op_lo;  // operand copies (hi, lo) of its grid charges
    const float *qlev;          // its cell charges
    float *loc;                 // its functionals (one kernel component)
};
// The launches (one per kernel component) of the cross-system tiles of a
// batch: levels lmin..lmax of every system, all cells.  sys: ncomp x nsys
// (component-major); depth: per system.  The lists and the per-system table
// are written to the device buffer *dx (grown as needed, owned by the caller).
int tc_cross_records(const std::vector<TcXSys> &sys, const std::vector<int> &depth, int ncomp, int lmin,
                     int lmax, int p3, int mode, int spow0, const void *const *k_hi_maps,
                     const void *const *k_lo_maps, const float *const *kbars, const WsLayout &W, int *status,
                     void **dx, size_t *dx_bytes, std::vector<LaunchRec> &out);
int launch_m2l_tc(const Geom &g, const Ptrs<float> &P, const WsLayout &W, const void *k_hi_map,
                  const void *k_lo_map, const float *kbar, int lmin, int mode, int inject,
                  float *loc, int spow, bool split, int comp, cudaStream_t st, Tracer &tr);
// map of a [343][p3s][pk] kernel table: fp32 (pk = p3s) or bf16 (pk = tc_padded_k)
int tc_encode_kernel_map(void *map, const void *base, int p3s, int pk, int mode);
int tc_padded(int p3);            // p^3 rounded up to 32 (MMA N, fp32 K)
int tc_padded_k(int p3, int mode);  // K extent of a cell vector: 32 (fp32) or 64 (bf16) multiple
size_t tc_map_bytes();

// bilinear forms without shifts (shift_free.cu, App. A.2; double-precision plans)
// table bytes and the first pair of every level (base[0..depth+1])
size_t sf_table_bytes(int p, int depth, int periodic, int64_t *base);
// allocates and computes the forms of every level (synchronous); also keeps
// the per-axis shift_{S->C} matrices of every level (hmat, offsets hoff)
int sf_build(int p, int depth, int periodic, const Coef<double> &C, void **tab, int64_t *base,
             void **hmat, int64_t *hoff);
// upward pass after the leaves' box-basis replacement: sums of children
void launch_sf_upward(const Geom &g, const Ptrs<double> &P, const WsLayout &W, cudaStream_t st,
                      Tracer &tr);
// interaction lists of every level plus the identity downward pass
void launch_sf_downward(const Geom &g, const Ptrs<double> &P, const WsLayout &W, const double *tab,
                        const int64_t *base, const double *hmat, const int64_t *hoff,
                        cudaStream_t st, Tracer &tr);

// the device a plan was created on (fmm_api.cu); the scratch array of
// fmm_eval_static on the current device, looked up once per device (fmm_static.cu)
int plan_device(const fmm_plan_s *plan);
int static_workspace_address(void **out);

// near field + far-field evaluation at the charges (kernels_p2p.cu)
// near field: writes out_pt (assigns) and the reaction slots; far field at the
// charges: adds them and the far field, stores the totals to out_e[perm[slot]]
template <typename real>
void launch_p2p(const Geom &g, const Ptrs<real> &P, const WsLayout &W, bool forces,
                cudaStream_t st, Tracer &tr);
template <typename real>
void launch_l2p(const Geom &g, const Coef<real> &C, const Ptrs<real> &P, const WsLayout &W,
                bool forces, cudaStream_t st, Tracer &tr);

}  // namespace fmm

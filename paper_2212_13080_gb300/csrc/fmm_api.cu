// C ABI of the GB300 replacement-FMM library: plans, tables, workspace layout
// and the order of the stages of one evaluation.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <new>
#include <type_traits>
#include <vector>

#include "fmm_internal.cuh"
#include "launch.cuh"

namespace fmm {
void far_set_attributes();

__global__ void __launch_bounds__(KZero::BS, KZero::MINB) k_zero_words(const __grid_constant__ KZero k) {
    k.run(blockIdx.x, gridDim.x);
}

void zero_words(Tracer &tr, int tag, void *p, size_t bytes, cudaStream_t st) {
    if (!tr.rec) {
        cudaMemsetAsync(p, 0, bytes, st);
        return;
    }
    const int64_t nw = (int64_t)(bytes / 4);
    const int blocks = (int)std::min<int64_t>(152 * 8, std::max<int64_t>(1, (nw + 4 * KZero::BS - 1) / (4 * KZero::BS)));
    launch_k(tr, tag, k_zero_words, KZero{reinterpret_cast<int *>(p), nw}, blocks, KZero::BS, 0, st);
}
}

using namespace fmm;

struct fmm_plan_s {
    long long id;  // distinct per plan (batched systems included): tags the workspace
    int depth, p, periodic;
    fmm_opts_t opts;
    double box[4];
    int64_t max_n;
    int device;
    bool fp64;
    // every table has ncomp blocks: the potential kernel 1/r and, with
    // FMM_FORCE_KERNEL, the three components of the force kernel r/|r|^3
    int ncomp;
    void *Kunit;  // [comp][343][p^3][p^3] Kt_o transposed ([o][b][a]), plan real type
    void *Kbar;   // [comp][343][p^3] row means of the unit-cell kernels
    void *Klat;   // [comp][p^3][p^3] lattice kernel minus its row mean (periodic form)
    void *Klbar;  // [comp][p^3] row means of the lattice kernel
    void *Ktc_hi, *Ktc_lo;  // [comp][343][a][b] split of Kt, padded (tensor-core plans)
    void *Kbar_tc;          // [comp][343][a] row means, padded to 32
    alignas(64) unsigned char khi_map[4][128], klo_map[4][128];  // their TMA tensor maps
    bool tc;                // bilinear forms of every level on tensor cores
    int tc_mode;            // FMM_TC_*: split TF32 x3, TF32 x1, split BF16 x3
    int inject;             // FMM_INJECT_* for the next evaluation (test hook)
    bool shared;            // tables belong to another plan (batched systems)
    void *sf_tab;           // App. A.2 forms of every level (shift-free plans), FP64
    int64_t sf_base[FMM_MAXDEPTH + 2];  // first pair of every level in sf_tab
    void *sf_H;             // per-axis shift_{S->C} of every level
    int64_t sf_hoff[FMM_MAXDEPTH + 2];
    Coef<float> cf;
    Coef<double> cd;
    Geom geom;
    const void *last_ws;
    int64_t last_n;
    int *h_hdr;  // pinned copy of the workspace header
    cudaStream_t s_near, s_coarse, s_far;  // auxiliary streams of an evaluation
    cudaEvent_t e_sorted, e_near, e_fork, e_coarse, e_far;
    bool timing;
    bool serial;  // timing mode 2: every stage on the call's stream
    cudaEvent_t ev[512];
    int nev_created;
    Tracer last;  // launches and stage events of the last call
};

static std::atomic<long long> g_plan_counter{0};

namespace fmm {
int plan_device(const fmm_plan_s *P) { return P->device; }
}  // namespace fmm

// Tag of an evaluation in the workspace header: plan id and n.
static long long eval_tag(const fmm_plan_s *P, int64_t n) { return (P->id << 32) | (long long)n; }

// ---------------------------------------------------------------------------
// FP64 tables (host)
// ---------------------------------------------------------------------------
namespace {

// §2.1.2: the p-division points of [0,1], i/(p-1); §4.1's reduced arrangement
// multiplies their spacing by gs <= 1 about the centre of the cell
double node(int p, double gs, int i) { return 0.5 + gs * ((double)i / (double)(p - 1) - 0.5); }

// §2.1.1: Lagrange basis g_i(x) on the p-division points of [0,1]
double lagrange(int p, double gs, int i, double x) {
    double v = 1.0;
    for (int k = 0; k < p; k++)
        if (k != i) v *= (x - node(p, gs, k)) / (node(p, gs, i) - node(p, gs, k));
    return v;
}

// Ewald-regularised sum over the lattice vectors m outside {-1,0,1}^3 of
// 1/|r + m| for r in [-1,1]^3 (unit cubic box, tin-foil boundary, neutralising
// background constant -pi/alpha^2): the Ewald pair potential of the unit box
// minus its 27 nearest image terms (§4.2, periodic form, level 0).
double far_image_sum(double rx, double ry, double rz);

// Its gradient, term by term (the force kernel of the lattice term is minus
// this): radial derivatives of -erf(a s)/s and erfc(a s)/s times (r + m)/s,
// and -4 pi w h sin(2 pi h.r) for each reciprocal pair.
void far_image_grad(double rx, double ry, double rz, double g[3]) {
    const double alpha = 2.0;
    const int RM = 7, HM = 7;
    const double c2 = 2.0 * alpha / std::sqrt(M_PI);
    g[0] = g[1] = g[2] = 0.0;
    for (int mz = -RM; mz <= RM; mz++)
        for (int my = -RM; my <= RM; my++)
            for (int mx = -RM; mx <= RM; mx++) {
                double x = rx + mx, y = ry + my, z = rz + mz;
                double s = std::sqrt(x * x + y * y + z * z);
                if (s == 0.0) continue;  // the near term is even and smooth at 0
                bool near = std::abs(mx) <= 1 && std::abs(my) <= 1 && std::abs(mz) <= 1;
                double e = c2 * std::exp(-alpha * alpha * s * s) / s;
                double d = near ? -e + std::erf(alpha * s) / (s * s) : -e - std::erfc(alpha * s) / (s * s);
                g[0] += d * x / s;
                g[1] += d * y / s;
                g[2] += d * z / s;
            }
    for (int hz = 0; hz <= HM; hz++)
        for (int hy = -HM; hy <= HM; hy++)
            for (int hx = -HM; hx <= HM; hx++) {
                if (hz == 0 && (hy < 0 || (hy == 0 && hx <= 0))) continue;
                double h2 = (double)(hx * hx + hy * hy + hz * hz);
                double w = std::exp(-M_PI * M_PI * h2 / (alpha * alpha)) / (M_PI * h2);
                double sn = std::sin(2.0 * M_PI * (hx * rx + hy * ry + hz * rz));
                g[0] -= 4.0 * M_PI * w * hx * sn;
                g[1] -= 4.0 * M_PI * w * hy * sn;
                g[2] -= 4.0 * M_PI * w * hz * sn;
            }
}

// The function of the bilinear forms between unit cells at separation
// (dx, dy, dz) = a - (o + b): comp 0 is 1/r (§2.1.7), comps 1..3 the x, y, z
// components of r/|r|^3 (§4.1: the forces directly from the kernel).
// power 2: 1/r^2 and the components of its force kernel 2 r/r^4 (§4.1 names
// 1/r^2 as another function the replacement applies to).
double kernel_value(int comp, int power, double dx, double dy, double dz) {
    const double r2 = dx * dx + dy * dy + dz * dz, r = std::sqrt(r2);
    const double d = comp == 1 ? dx : comp == 2 ? dy : dz;
    if (power == 2) return comp == 0 ? 1.0 / r2 : 2.0 * d / (r2 * r2);
    return comp == 0 ? 1.0 / r : d / (r2 * r);
}

double far_image_sum(double rx, double ry, double rz) {
    const double alpha = 2.0;
    const int RM = 7, HM = 7;
    const double spi = std::sqrt(M_PI);
    double real_part = 0.0;
    for (int mz = -RM; mz <= RM; mz++)
        for (int my = -RM; my <= RM; my++)
            for (int mx = -RM; mx <= RM; mx++) {
                double x = rx + mx, y = ry + my, z = rz + mz;
                double s = std::sqrt(x * x + y * y + z * z);
                bool near = std::abs(mx) <= 1 && std::abs(my) <= 1 && std::abs(mz) <= 1;
                if (near) {
                    // erfc(as)/s - 1/s = -erf(as)/s, -> -2a/sqrt(pi) at s = 0
                    real_part += (s > 0.0) ? -std::erf(alpha * s) / s : -2.0 * alpha / spi;
                } else {
                    real_part += std::erfc(alpha * s) / s;
                }
            }
    double recip = 0.0;
    for (int hz = 0; hz <= HM; hz++)
        for (int hy = -HM; hy <= HM; hy++)
            for (int hx = -HM; hx <= HM; hx++) {
                // half space hz > 0, plus hz == 0 with (hy, hx) > 0; pairs +-h
                if (hz == 0 && (hy < 0 || (hy == 0 && hx <= 0))) continue;
                double h2 = (double)(hx * hx + hy * hy + hz * hz);
                double w = std::exp(-M_PI * M_PI * h2 / (alpha * alpha)) / (M_PI * h2);
                recip += 2.0 * w * std::cos(2.0 * M_PI * (hx * rx + hy * ry + hz * rz));
            }
    return real_part + recip - M_PI / (alpha * alpha);
}

template <typename real>
void fill_coef(int p, double gs, Coef<real> &C) {
    memset(&C, 0, sizeof(C));
    for (int i = 0; i < p; i++) {
        C.tau[i] = (real)node(p, gs, i);
        double den = 1.0;
        for (int k = 0; k < p; k++)
            if (k != i) den *= node(p, gs, i) - node(p, gs, k);
        C.cinv[i] = (real)(1.0 / den);
    }
    // eq. (trans): (J,i) entry = parent basis g_J at the child node (h + tau_i)/2
    for (int h = 0; h < 2; h++)
        for (int J = 0; J < p; J++)
            for (int i = 0; i < p; i++) C.G[h][J * p + i] = (real)lagrange(p, gs, J, 0.5 * (h + node(p, gs, i)));
}

template <typename real>
int upload(void **dst, const std::vector<real> &v) {
    if (cudaMalloc(dst, v.size() * sizeof(real)) != cudaSuccess) return FMM_ERR_OOM;
    if (cudaMemcpy(*dst, v.data(), v.size() * sizeof(real), cudaMemcpyHostToDevice) != cudaSuccess)
        return FMM_ERR_CUDA;
    return FMM_OK;
}

// bfloat16 = the upper 16 bits of an IEEE binary32; round to nearest, ties to
// even, on the discarded 16 bits (finite inputs only)
static uint16_t bf16_rne(float f) {
    uint32_t u;
    memcpy(&u, &f, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}
static float bf16_value(uint16_t h) {
    uint32_t u = (uint32_t)h << 16;
    float f;
    memcpy(&f, &u, 4);
    return f;
}

// Unit-cell kernels of eq. (bilinear), K_o[a,b] = 1/|a - (o + b)| for the 316
// offsets 2 <= |o|_inf <= 3 (and, with FMM_FORCE_KERNEL, the three force
// kernels), split into row mean and remainder (FP64, then rounded to the
// plan's type).
template <typename real>
int upload_tables(fmm_plan_t P) {
    const int p = P->p, p3 = p * p * p, nc = P->ncomp, pw = P->geom.power;
    const double gs = P->opts.grid_scale;
    const size_t nk = (size_t)343 * p3 * p3;
    std::vector<real> KtT(nc * nk, (real)0), Kbar((size_t)nc * 343 * p3, (real)0);
    std::vector<double> row(p3);
    for (int c = 0; c < nc; c++)
        for (int oz = -3; oz <= 3; oz++)
            for (int oy = -3; oy <= 3; oy++)
                for (int ox = -3; ox <= 3; ox++) {
                    if (std::abs(ox) <= 1 && std::abs(oy) <= 1 && std::abs(oz) <= 1) continue;
                    size_t oi = (size_t)c * 343 + (size_t)(((oz + 3) * 7 + (oy + 3)) * 7 + (ox + 3));
                    for (int a = 0; a < p3; a++) {
                        double ax = node(p, gs, a % p), ay = node(p, gs, (a / p) % p), az = node(p, gs, a / (p * p));
                        double mean = 0.0;
                        for (int b = 0; b < p3; b++) {
                            row[b] = kernel_value(c, pw, ax - (ox + node(p, gs, b % p)),
                                                  ay - (oy + node(p, gs, (b / p) % p)),
                                                  az - (oz + node(p, gs, b / (p * p))));
                            mean += row[b];
                        }
                        mean /= p3;
                        Kbar[oi * p3 + a] = (real)mean;
                        for (int b = 0; b < p3; b++) KtT[(oi * p3 + b) * p3 + a] = (real)(row[b] - mean);
                    }
                }
    int rc = upload(&P->Kunit, KtT);
    if (!rc) rc = upload(&P->Kbar, Kbar);
    if (rc) return rc;
    if (P->tc) {
        // Kt_o[a][b] = K_o[a][b] - Kbar_o[a] (natural layout, rows zero-padded to
        // p3s = p^3 rounded up to 32, columns to pk), split from the FP64 value:
        // TF32: hi = Kt with its 13 low mantissa bits cleared (rounded to nearest
        // for the 1-pass form), lo = Kt - hi;
        // BF16: hi = bf16(Kt), lo = bf16(Kt - hi), rounded to nearest even
        const int p3s = tc_padded(p3), pk = tc_padded_k(p3, P->tc_mode);
        const bool bf16 = P->tc_mode == FMM_TC_BF16X3;
        const size_t nt = (size_t)343 * p3s * pk;
        std::vector<float> Khi(nc * nt, 0.0f), Klo(nc * nt, 0.0f), Kb((size_t)nc * 343 * p3s, 0.0f);
        std::vector<uint16_t> Khi16(bf16 ? nc * nt : 0, 0), Klo16(bf16 ? nc * nt : 0, 0);
        for (int oc = 0; oc < 343 * nc; oc++) {
            const int c = oc / 343, oi = oc % 343;
            int ox = oi % 7 - 3, oy = (oi / 7) % 7 - 3, oz = oi / 49 - 3;
            if (std::abs(ox) <= 1 && std::abs(oy) <= 1 && std::abs(oz) <= 1) continue;
            for (int a = 0; a < p3; a++) {
                double ax = node(p, gs, a % p), ay = node(p, gs, (a / p) % p), az = node(p, gs, a / (p * p));
                double mean = 0.0;
                for (int b = 0; b < p3; b++) {
                    row[b] = kernel_value(c, pw, ax - (ox + node(p, gs, b % p)), ay - (oy + node(p, gs, (b / p) % p)),
                                          az - (oz + node(p, gs, b / (p * p))));
                    mean += row[b];
                }
                mean /= p3;
                Kb[(size_t)oc * p3s + a] = (float)mean;
                for (int b = 0; b < p3; b++) {
                    double k = row[b] - mean;
                    size_t idx = ((size_t)oc * p3s + a) * pk + b;
                    if (bf16) {
                        uint16_t h = bf16_rne((float)k);
                        Khi16[idx] = h;
                        Klo16[idx] = bf16_rne((float)(k - (double)bf16_value(h)));
                        continue;
                    }
                    float f = (float)k;
                    uint32_t u;
                    memcpy(&u, &f, 4);
                    if (P->tc_mode == FMM_TC_TF32X1) u += 0x1000u;  // nearest (no lo pass)
                    u &= 0xFFFFE000u;
                    float hi;
                    memcpy(&hi, &u, 4);
                    Khi[idx] = hi;
                    Klo[idx] = (float)(k - (double)hi);
                }
            }
        }
        rc = bf16 ? upload(&P->Ktc_hi, Khi16) : upload(&P->Ktc_hi, Khi);
        if (!rc) rc = bf16 ? upload(&P->Ktc_lo, Klo16) : upload(&P->Ktc_lo, Klo);
        if (!rc) rc = upload(&P->Kbar_tc, Kb);
        const size_t cb = nt * (bf16 ? 2 : 4);  // bytes of one component's table
        for (int c = 0; c < nc && !rc; c++) {
            rc = tc_encode_kernel_map(P->khi_map[c], (const char *)P->Ktc_hi + c * cb, p3s, pk, P->tc_mode);
            if (!rc) rc = tc_encode_kernel_map(P->klo_map[c], (const char *)P->Ktc_lo + c * cb, p3s, pk, P->tc_mode);
        }
        if (rc) return rc;
    }
    if (P->periodic) {
        // psi depends on a - b only: (2p-1)^3 distinct arguments; the force
        // components take -grad psi
        const int m = 2 * p - 1;
        std::vector<double> tab((size_t)nc * m * m * m);
        for (int dz = 0; dz < m; dz++)
            for (int dy = 0; dy < m; dy++)
                for (int dx = 0; dx < m; dx++) {
                    const double rx = gs * (dx - (p - 1)) / (double)(p - 1),
                                 ry = gs * (dy - (p - 1)) / (double)(p - 1),
                                 rz = gs * (dz - (p - 1)) / (double)(p - 1);
                    const size_t e = ((size_t)dz * m + dy) * m + dx;
                    tab[e] = far_image_sum(rx, ry, rz);
                    if (nc > 1) {
                        double gr[3];
                        far_image_grad(rx, ry, rz, gr);
                        for (int c = 1; c < nc; c++) tab[(size_t)c * m * m * m + e] = -gr[c - 1];
                    }
                }
        std::vector<real> Kl((size_t)nc * p3 * p3), Klb((size_t)nc * p3);
        for (int c = 0; c < nc; c++)
            for (int a = 0; a < p3; a++) {
                double mean = 0.0;
                for (int b = 0; b < p3; b++) {
                    int dx = a % p - b % p + p - 1, dy = (a / p) % p - (b / p) % p + p - 1,
                        dz = a / (p * p) - b / (p * p) + p - 1;
                    row[b] = tab[(size_t)c * m * m * m + ((size_t)dz * m + dy) * m + dx];
                    mean += row[b];
                }
                mean /= p3;
                Klb[(size_t)c * p3 + a] = (real)mean;
                for (int b = 0; b < p3; b++) Kl[((size_t)c * p3 + a) * p3 + b] = (real)(row[b] - mean);
            }
        rc = upload(&P->Klat, Kl);
        if (!rc) rc = upload(&P->Klbar, Klb);
        if (rc) return rc;
    }
    return FMM_OK;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

WsLayout make_layout(const fmm_plan_t P, int64_t n) {
    WsLayout W;
    memset(&W, 0, sizeof(W));
    const size_t rs = P->fp64 ? 8 : 4;
    const int p3 = P->p * P->p * P->p;
    const bool cont = P->opts.continuous != 0;
    W.ncell = (int64_t)1 << (3 * P->depth);
    if (cont) {
        // default: 1.5x the expected charges per particle for uniform density,
        // (1 + 2 d/w (m - 1))^3 with m charges per split axis, and at least 2
        const int m = P->p + (P->p & 1);
        double e1 = 1.0 + 2.0 * P->opts.split_ratio * (m - 1);
        double fdef = 1.5 * e1 * e1 * e1;
        if (fdef < 2.0) fdef = 2.0;
        double f = P->opts.split_capacity > 0 ? P->opts.split_capacity : fdef;
        W.cap = (int64_t)std::ceil(f * (double)n) + 64;
        if (W.cap < n) W.cap = n;
    } else {
        W.cap = n;
    }
    if (W.cap < 1) W.cap = 1;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t r = o;
        o += align256(bytes);
        return r;
    };
    W.hdr = take(256);
    W.count = take(cont ? n * 4 : 0);
    W.offset = take(cont ? (n + 1) * 4 : 0);
    W.axes = take(cont ? n : 0);
    W.e_key = take(W.cap * 4);
    W.e_pt = take(W.cap * 4 * rs);
    W.e_wd = take(cont ? W.cap * 4 * rs : 0);
    W.e_origin = take(W.cap * 4);
    W.e_rank = take(W.cap * 4);
    W.leaf_count = take(W.ncell * 4);
    W.leaf_start = take((W.ncell + 1) * 4);
    W.tmp = take(W.cap * 4);
    W.perm = take(W.cap * 4);
    W.s_pt = take(W.cap * 4 * rs);
    W.s_origin = take(W.cap * 4);
    W.out_pt = take(W.cap * 4 * rs);
    W.react = take(13 * W.cap * 4 * rs);
    int64_t ph = 0, lc = 0;
    for (int l = 0; l <= P->depth; l++) {
        W.phi_level[l] = ph * p3;
        W.loc_level[l] = lc * p3;
        ph += phi_level_cells(l);
        lc += loc_level_cells(l);
    }
    W.phi_level[P->depth + 1] = ph * p3;
    W.loc_level[P->depth + 1] = lc * p3;
    W.phi = take((size_t)ph * p3 * rs);
    W.loc_comp = lc * p3;  // functionals of one kernel component
    W.loc = take((size_t)lc * p3 * rs * P->ncomp);
    int64_t qc = 0;
    for (int l = 0; l <= P->depth; l++) {
        W.q_level[l] = qc;
        qc += phi_level_cells(l);
    }
    W.q_level[P->depth + 1] = qc;
    W.qlev = take((size_t)qc * rs);
    size_t part = 0;
    for (int l = 2; l <= P->depth; l++) {
        int G = m2l_groups(l, p3);
        if (G > 1) {
            size_t need = (size_t)G * ((size_t)1 << (3 * l)) * p3;
            if (need > part) part = need;
        }
    }
    if (P->periodic) {
        int G = m2l_groups(1, p3);
        size_t need = (size_t)G * 8 * p3;
        if (G > 1 && need > part) part = need;
    }
    W.m2l_part = take(part * rs);
    const size_t p3s = (size_t)tc_padded(p3);
    const size_t pht = (size_t)tc_level_first(P->depth + 1);  // cells of the operand layout
    W.phihi = take(P->tc ? pht * p3s * rs : 0);
    W.philo = take(P->tc ? pht * p3s * rs : 0);
    W.occ = take(P->tc ? (size_t)occ_ints(P->depth, P->periodic ? 1 : 2) * 4 : 0);
    W.delta = take(cont && !P->fp64 ? (size_t)W.cap * 4 : 0);
    W.slist = take(cont && !P->fp64 ? (size_t)(n + 2) * 4 : 0);
    W.pord = take((size_t)(W.ncell + 16) * 4);
    int64_t mx = n > W.ncell ? n : W.ncell;
    W.scan_blocks = (int)(mx / 2048 + 2);
    W.scan_tmp = take((size_t)(W.scan_blocks + 1) * 4);
    W.epart = take((size_t)((n + 255) / 256 + 1) * 16);  // (hi, lo) per block, real <= 8 B
    W.total = o;
    return W;
}

template <typename real>
Ptrs<real> make_ptrs(const WsLayout &W, void *ws) {
    char *b = (char *)ws;
    Ptrs<real> P;
    typedef typename Vec4<real>::T R4;
    P.hdr = (WsHeader *)(b + W.hdr);
    P.count = (int *)(b + W.count);
    P.offset = (int *)(b + W.offset);
    P.axes = (unsigned char *)(b + W.axes);
    P.e_key = (uint32_t *)(b + W.e_key);
    P.e_pt = (R4 *)(b + W.e_pt);
    P.e_wd = (R4 *)(b + W.e_wd);
    P.e_origin = (int *)(b + W.e_origin);
    P.e_rank = (int *)(b + W.e_rank);
    P.leaf_count = (int *)(b + W.leaf_count);
    P.leaf_start = (int *)(b + W.leaf_start);
    P.tmp = (int *)(b + W.tmp);
    P.perm = (int *)(b + W.perm);
    P.s_pt = (R4 *)(b + W.s_pt);
    P.s_origin = (int *)(b + W.s_origin);
    P.out_pt = (R4 *)(b + W.out_pt);
    P.out_e = P.e_pt;  // e_pt is dead once the sort has gathered it
    P.react = (R4 *)(b + W.react);
    P.phi = (real *)(b + W.phi);
    P.loc = (real *)(b + W.loc);
    P.qlev = (real *)(b + W.qlev);
    P.m2l_part = (real *)(b + W.m2l_part);
    P.phihi = (real *)(b + W.phihi);
    P.philo = (real *)(b + W.philo);
    P.occ = (int *)(b + W.occ);
    P.delta = (float *)(b + W.delta);
    P.slist = (int *)(b + W.slist);
    P.pord = (int *)(b + W.pord);
    P.scan_tmp = (int *)(b + W.scan_tmp);
    P.epart = (double *)(b + W.epart);
    return P;
}

int status_to_error(int st) {
    if (st & ST_STATE) return FMM_ERR_STATE;
    if (st & ST_TIMEOUT) return FMM_ERR_TIMEOUT;
    if (st & ST_NONFINITE) return FMM_ERR_NONFINITE;
    if (st & ST_OUT_OF_BOX) return FMM_ERR_OUT_OF_BOX;
    if (st & ST_SPLIT_OVERFLOW) return FMM_ERR_SPLIT_OVERFLOW;
    return FMM_OK;
}

struct KMarkValid {
    static constexpr int BS = 32, MINB = 1;
    WsHeader *hdr;
    long long tag;
    __device__ void run(int, int) const {
        if (threadIdx.x == 0) {
            hdr->valid = 1;
            hdr->tag = tag;
        }
    }
};
__global__ void __launch_bounds__(KMarkValid::BS, KMarkValid::MINB) k_mark_valid(const __grid_constant__ KMarkValid k) {
    k.run(blockIdx.x, gridDim.x);
}

// the backward pass reuses the state of the last evaluation on the workspace:
// it must be this plan's, for this n
__global__ void k_check_state(WsHeader *hdr, long long tag) {
    if (!hdr->valid || hdr->tag != tag) atomicOr(&hdr->status, ST_STATE);
}

int check_ws(const fmm_plan_t P, int64_t n, const void *ws, size_t bytes) {
    if (!ws) return FMM_ERR_WORKSPACE;
    if (((uintptr_t)ws) & 255) return FMM_ERR_WORKSPACE;
    WsLayout W = make_layout(P, n);
    if (bytes < W.total) return FMM_ERR_WORKSPACE;
    return FMM_OK;
}

int finish(fmm_plan_t P, const WsHeader *hdr, cudaStream_t st, bool sync) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return FMM_ERR_CUDA;
    if (!sync) return FMM_OK;
    if (cudaMemcpyAsync(P->h_hdr, hdr, sizeof(WsHeader), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return FMM_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return FMM_ERR_CUDA;
    return status_to_error(P->h_hdr[0]);
}

template <typename real>
int eval_impl(fmm_plan_t P, int64_t n, const float *pos, const float *q, real *potential,
              double *energy, real *forces, void *ws, const Streams &S, Tracer &tr) {
    cudaStream_t st = S.main;
    WsLayout W = make_layout(P, n);
    Ptrs<real> ptr = make_ptrs<real>(W, ws);
    const Coef<real> &C = *reinterpret_cast<const Coef<real> *>(P->fp64 ? (const void *)&P->cd
                                                                        : (const void *)&P->cf);
    Geom g = P->geom;
    zero_words(tr, FMM_TAG(S_ZERO_HDR, 0), ptr.hdr, 256, st);
    if (n == 0) {
        launch_unsplit<real>(g, ptr, W, 0, q, potential, energy, forces, nullptr, nullptr, false, st,
                             tr);
        return FMM_OK;
    }
    zero_words(tr, FMM_TAG(S_ZERO_LEAF, 0), ptr.leaf_count, W.ncell * 4, st);
    launch_bin_emit<real>(g, C, ptr, W, (int)n, pos, q, st, tr);
    launch_sort<real>(g, ptr, W, (int)n, st, tr);
    // the near field needs only the sorted charges: it runs on its own stream
    // beside the whole far field and joins before the far field is added
    // (recorded launches: the near stream's are marked, the join is a marker)
    if (!tr.rec) {
        cudaEventRecord(S.sorted, st);
        cudaStreamWaitEvent(S.near, S.sorted, 0);
    }
    tr.near = S.near;
    launch_p2p<real>(g, ptr, W, forces != nullptr, S.near, tr);
    tr.near = nullptr;
    if (!tr.rec) cudaEventRecord(S.near_done, S.near);
    // the far field runs on a high-priority stream when one is given, so that
    // its CTAs are dispatched ahead of the near field's as SMs free up
    Streams F = S;
    if (S.far && !tr.rec) {
        cudaStreamWaitEvent(S.far, S.sorted, 0);
        F.main = S.far;
    }
    launch_upward<real>(g, C, ptr, W, F.main, tr);
    DevTables<real> T;
    const int p3 = g.p3;
    T.ncomp = P->ncomp;
    for (int c = 0; c < P->ncomp; c++) {
        T.KtT[c] = (const real *)P->Kunit + (size_t)c * 343 * p3 * p3;
        T.Kbar[c] = (const real *)P->Kbar + (size_t)c * 343 * p3;
        T.Klt[c] = P->Klat ? (const real *)P->Klat + (size_t)c * p3 * p3 : nullptr;
        T.Klbar[c] = P->Klbar ? (const real *)P->Klbar + (size_t)c * p3 : nullptr;
        T.tc_khi_map[c] = P->khi_map[c];
        T.tc_klo_map[c] = P->klo_map[c];
        T.tc_kbar[c] = P->Kbar_tc ? (const float *)P->Kbar_tc + (size_t)c * 343 * tc_padded(p3) : nullptr;
    }
    T.tc_lmin = P->tc ? (P->periodic ? 1 : 2) : 0;  // every level on the tensor cores
    T.tc_mode = P->tc_mode;
    T.tc_inject = P->inject;
    P->inject = FMM_INJECT_NONE;  // one evaluation only
    T.sf_tab = (const double *)P->sf_tab;
    T.sf_base = P->sf_base;
    T.sf_H = (const double *)P->sf_H;
    T.sf_hoff = P->sf_hoff;
    int rc = launch_downward<real>(g, C, ptr, W, T, F, tr);
    if (rc) return rc;
    if constexpr (std::is_same<real, float>::value)
        if (g.continuous && forces && g.force_mode == FMM_FORCE_ADJOINT)
            launch_split_delta(g, P->cd, ptr, W, (int)n, pos, F.main, tr);
    if (S.far && !tr.rec) {
        cudaEventRecord(S.far_done, S.far);
        cudaStreamWaitEvent(st, S.far_done, 0);
    }
    if (!tr.rec) cudaStreamWaitEvent(st, S.near_done, 0);
    else record_marker(tr, FMM_TAG(S_JOIN_NEAR, 0));
    launch_l2p<real>(g, C, ptr, W, forces != nullptr, st, tr);
    launch_unsplit<real>(g, ptr, W, (int)n, q, potential, energy, forces, nullptr, nullptr, false,
                         st, tr);
    launch_k(tr, FMM_TAG(S_MARK_VALID, 0), k_mark_valid, KMarkValid{ptr.hdr, eval_tag(P, n)}, 1, KMarkValid::BS, 0,
             st);
    tr.count();
    return FMM_OK;
}

template <typename real>
int backward_impl(fmm_plan_t P, int64_t n, const float *pos, const float *q, const double *gE, real *grad_pos,
                  real *grad_q, void *ws, cudaStream_t st, Tracer &tr) {
    WsLayout W = make_layout(P, n);
    Ptrs<real> ptr = make_ptrs<real>(W, ws);
    const Coef<real> &C = *reinterpret_cast<const Coef<real> *>(P->fp64 ? (const void *)&P->cd
                                                                        : (const void *)&P->cf);
    Geom g = P->geom;
    if (n == 0) return FMM_OK;
    k_check_state<<<1, 1, 0, st>>>(ptr.hdr, eval_tag(P, n));
    tr.count();
    // the gradient of the energy: adjoint forces whatever the forward mode
    if (g.force_mode == FMM_FORCE_KERNEL) g.force_mode = FMM_FORCE_ADJOINT;
    launch_p2p<real>(g, ptr, W, true, st, tr);
    launch_l2p<real>(g, C, ptr, W, true, st, tr);
    if constexpr (std::is_same<real, float>::value)
        if (g.continuous && g.force_mode == FMM_FORCE_ADJOINT)
            launch_split_delta(g, P->cd, ptr, W, (int)n, pos, st, tr);
    launch_unsplit<real>(g, ptr, W, (int)n, q, nullptr, nullptr, grad_pos, gE, grad_q, true, st, tr);
    return FMM_OK;
}

Tracer make_tracer(fmm_plan_t P, cudaStream_t st) {
    Tracer tr;
    tr.st = st;
    tr.on = P->timing;
    tr.ev = P->ev;
    tr.cap = P->nev_created;
    return tr;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

void fmm_opts_default(fmm_opts_t *o) {
    if (!o) return;
    o->continuous = 0;
    o->split_ratio = 1.0 / 256.0;
    o->split_capacity = 0.0;
    o->precision = FMM_PREC_FP32;
    o->force_mode = FMM_FORCE_ADJOINT;
    o->sync = 1;
    o->grid_scale = 1.0;
    o->shift_free = 0;
    o->kernel = FMM_KERNEL_COULOMB;
}

const char *fmm_strerror(int s) {
    switch (s) {
    case FMM_OK: return "ok";
    case FMM_ERR_ARG: return "invalid argument";
    case FMM_ERR_OOM: return "out of device memory";
    case FMM_ERR_OUT_OF_BOX: return "position outside the box (open form)";
    case FMM_ERR_NONFINITE: return "non-finite position";
    case FMM_ERR_SPLIT_OVERFLOW: return "more split charges than the workspace holds";
    case FMM_ERR_TIMEOUT: return "device wait timed out";
    case FMM_ERR_CUDA: return "CUDA runtime error";
    case FMM_ERR_STATE: return "no evaluation to differentiate";
    case FMM_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    case FMM_ERR_UNSUPPORTED: return "unsupported configuration";
    default: return "unknown status";
    }
}

int fmm_version(void) { return 100; }

int fmm_plan_create(fmm_plan_t *out, const double box[4], int depth, int p, int periodic,
                    const fmm_opts_t *opts, int64_t max_n) {
    if (!out || !box) return FMM_ERR_ARG;
    *out = nullptr;
    if (depth < 2 || depth > FMM_MAXDEPTH || p < 2 || p > FMM_MAXP) return FMM_ERR_ARG;
    if (!(box[3] > 0.0) || !std::isfinite(box[0]) || !std::isfinite(box[1]) ||
        !std::isfinite(box[2]) || !std::isfinite(box[3]))
        return FMM_ERR_ARG;
    if (max_n < 0 || max_n > (int64_t)1 << 30) return FMM_ERR_ARG;
    fmm_opts_t o;
    fmm_opts_default(&o);
    if (opts) o = *opts;
    if (o.split_ratio <= 0) o.split_ratio = 1.0 / 256.0;
    if (o.grid_scale <= 0) o.grid_scale = 1.0;
    if (!(o.grid_scale <= 1.0)) return FMM_ERR_ARG;
    // the split weights (§2.3) are Lagrange weights on equally spaced segment
    // nodes: the reduced arrangement is for the plain form
    if (o.continuous && o.grid_scale != 1.0) return FMM_ERR_UNSUPPORTED;
    if (o.continuous && !(o.split_ratio < 0.5)) return FMM_ERR_ARG;
    if (o.force_mode != FMM_FORCE_ADJOINT && o.force_mode != FMM_FORCE_PAPER &&
        o.force_mode != FMM_FORCE_KERNEL)
        return FMM_ERR_ARG;
    if (o.force_mode == FMM_FORCE_KERNEL && o.shift_free) return FMM_ERR_UNSUPPORTED;
    if (o.kernel != FMM_KERNEL_COULOMB && o.kernel != FMM_KERNEL_INV_SQUARE) return FMM_ERR_ARG;
    // the lattice sum of 1/r^2 diverges; the shift-free forms are built for 1/r
    if (o.kernel == FMM_KERNEL_INV_SQUARE && (periodic || o.shift_free)) return FMM_ERR_UNSUPPORTED;
    const bool tc_prec = o.precision == FMM_PREC_TF32X3 || o.precision == FMM_PREC_TF32X1 ||
                         o.precision == FMM_PREC_BF16X3;
    if (o.precision != FMM_PREC_FP32 && o.precision != FMM_PREC_FP64 && !tc_prec)
        return FMM_ERR_UNSUPPORTED;
    if (tc_prec && (p < 3 || p > 6)) return FMM_ERR_UNSUPPORTED;
    // App. A.2 forms: FP64 (they extrapolate over 2^l cells), p <= 5, <= 32 GiB
    if (o.shift_free) {
        int64_t base[FMM_MAXDEPTH + 2];
        if (o.precision != FMM_PREC_FP64 || p > 5 || o.grid_scale != 1.0 ||
            fmm::sf_table_bytes(p, depth, periodic ? 1 : 0, base) > ((size_t)32 << 30))
            return FMM_ERR_UNSUPPORTED;
    }
    fmm_plan_s *P = new (std::nothrow) fmm_plan_s();
    if (!P) return FMM_ERR_OOM;
    P->id = ++g_plan_counter;
    P->depth = depth;
    P->p = p;
    P->periodic = periodic ? 1 : 0;
    P->opts = o;
    P->ncomp = o.force_mode == FMM_FORCE_KERNEL ? 4 : 1;
    memcpy(P->box, box, sizeof(double) * 4);
    P->max_n = max_n;
    P->fp64 = o.precision == FMM_PREC_FP64;
    P->tc = tc_prec;
    P->tc_mode = o.precision == FMM_PREC_BF16X3   ? FMM_TC_BF16X3
                 : o.precision == FMM_PREC_TF32X1 ? FMM_TC_TF32X1
                                                  : FMM_TC_TF32X3;
    cudaGetDevice(&P->device);
    fill_coef<float>(p, o.grid_scale, P->cf);
    fill_coef<double>(p, o.grid_scale, P->cd);
    Geom &g = P->geom;
    g.p = p;
    g.p3 = p * p * p;
    g.depth = depth;
    g.periodic = P->periodic;
    g.continuous = o.continuous ? 1 : 0;
    g.force_mode = o.force_mode;
    g.shift_free = o.shift_free ? 1 : 0;
    g.power = o.kernel == FMM_KERNEL_INV_SQUARE ? 2 : 1;
    g.S = 1 << depth;
    for (int a = 0; a < 3; a++) g.x0[a] = (float)box[a];
    g.Lf = (float)box[3];
    g.dtf = (float)o.split_ratio;
    g.dthi = 1.0f - g.dtf;
    g.L = box[3];
    if (cudaMallocHost(&P->h_hdr, 256) != cudaSuccess) {
        delete P;
        return FMM_ERR_OOM;
    }
    {
        int lo = 0, hi = 0;
        cudaDeviceGetStreamPriorityRange(&lo, &hi);
        // near field: lowest priority (it fills the GPU); coarse levels: highest
        if (cudaStreamCreateWithPriority(&P->s_near, cudaStreamNonBlocking, lo) != cudaSuccess ||
            cudaStreamCreateWithPriority(&P->s_coarse, cudaStreamNonBlocking, hi) != cudaSuccess ||
            cudaStreamCreateWithPriority(&P->s_far, cudaStreamNonBlocking, hi) != cudaSuccess ||
            cudaEventCreateWithFlags(&P->e_far, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&P->e_sorted, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&P->e_near, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&P->e_fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&P->e_coarse, cudaEventDisableTiming) != cudaSuccess) {
            fmm_plan_destroy(P);
            return FMM_ERR_CUDA;
        }
    }
    fmm::far_set_attributes();
    int rc = P->fp64 ? upload_tables<double>(P) : upload_tables<float>(P);
    if (rc == FMM_OK && o.shift_free) rc = fmm::sf_build(p, depth, P->periodic, P->cd, &P->sf_tab, P->sf_base, &P->sf_H,
                                                   P->sf_hoff);
    // the tables went up by cudaMemcpy from pageable memory, which may return
    // before the transfer lands; an evaluation on a non-blocking stream is not
    // ordered after it
    if (rc == FMM_OK && cudaDeviceSynchronize() != cudaSuccess) rc = FMM_ERR_CUDA;
    if (rc != FMM_OK) {
        fmm_plan_destroy(P);
        return rc;
    }
    *out = P;
    return FMM_OK;
}

void fmm_plan_destroy(fmm_plan_t P) {
    if (!P) return;
    if (P->shared) {
        delete P;
        return;
    }
    if (P->s_near) cudaStreamDestroy(P->s_near);
    if (P->s_coarse) cudaStreamDestroy(P->s_coarse);
    if (P->s_far) cudaStreamDestroy(P->s_far);
    if (P->e_far) cudaEventDestroy(P->e_far);
    if (P->e_sorted) cudaEventDestroy(P->e_sorted);
    if (P->e_near) cudaEventDestroy(P->e_near);
    if (P->e_fork) cudaEventDestroy(P->e_fork);
    if (P->e_coarse) cudaEventDestroy(P->e_coarse);
    for (int i = 0; i < P->nev_created; i++) cudaEventDestroy(P->ev[i]);
    if (P->Kunit) cudaFree(P->Kunit);
    if (P->Kbar) cudaFree(P->Kbar);
    if (P->Klat) cudaFree(P->Klat);
    if (P->Klbar) cudaFree(P->Klbar);
    if (P->Ktc_hi) cudaFree(P->Ktc_hi);
    if (P->Ktc_lo) cudaFree(P->Ktc_lo);
    if (P->Kbar_tc) cudaFree(P->Kbar_tc);
    if (P->sf_tab) cudaFree(P->sf_tab);
    if (P->sf_H) cudaFree(P->sf_H);
    if (P->h_hdr) cudaFreeHost(P->h_hdr);
    delete P;
}

int fmm_workspace_size(fmm_plan_t P, int64_t n, size_t *bytes) {
    if (!P || !bytes || n < 0 || n > P->max_n) return FMM_ERR_ARG;
    *bytes = make_layout(P, n).total;
    return FMM_OK;
}

int fmm_eval(fmm_plan_t P, int64_t n, const float *pos, const float *q, void *potential,
             double *energy, void *forces, void *workspace, size_t workspace_bytes, void *stream) {
    if (!P || n < 0 || n > P->max_n) return FMM_ERR_ARG;
    if (n > 0 && (!pos || !q)) return FMM_ERR_ARG;
    int rc = check_ws(P, n, workspace, workspace_bytes);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    cudaGetLastError();
    if (P->opts.sync) {  // the final wait would end a capture in progress
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return FMM_ERR_CUDA;
        if (cs != cudaStreamCaptureStatusNone) return FMM_ERR_ARG;
    }
    Tracer tr = make_tracer(P, st);
    Streams S = {st, P->s_near, P->s_coarse, P->e_sorted, P->e_near, P->e_fork, P->e_coarse,
                 P->s_far, P->e_far};
    if (P->serial) S.near = S.coarse = st, S.far = nullptr;  // isolated stage times
    if (P->fp64)
        rc = eval_impl<double>(P, n, pos, q, (double *)potential, energy, (double *)forces, workspace, S, tr);
    else
        rc = eval_impl<float>(P, n, pos, q, (float *)potential, energy, (float *)forces, workspace, S, tr);
    P->last = tr;
    if (rc) return rc;
    P->last_ws = workspace;
    P->last_n = n;
    WsLayout W = make_layout(P, n);
    return finish(P, (const WsHeader *)((char *)workspace + W.hdr), st, P->opts.sync != 0);
}

int fmm_backward(fmm_plan_t P, int64_t n, const float *pos, const float *q,
                 const double *grad_energy, void *grad_pos, void *grad_q, void *workspace,
                 size_t workspace_bytes, void *stream) {
    if (!P || n < 0 || n > P->max_n || !grad_energy) return FMM_ERR_ARG;
    if (n > 0 && (!q || !pos)) return FMM_ERR_ARG;
    int rc = check_ws(P, n, workspace, workspace_bytes);
    if (rc) return rc;
    if (P->last_ws != workspace || P->last_n != n) return FMM_ERR_STATE;
    cudaStream_t st = (cudaStream_t)stream;
    cudaGetLastError();
    Tracer tr = make_tracer(P, st);
    if (P->fp64)
        rc = backward_impl<double>(P, n, pos, q, grad_energy, (double *)grad_pos, (double *)grad_q, workspace, st, tr);
    else
        rc = backward_impl<float>(P, n, pos, q, grad_energy, (float *)grad_pos, (float *)grad_q, workspace, st, tr);
    P->last = tr;
    if (rc) return rc;
    WsLayout W = make_layout(P, n);
    return finish(P, (const WsHeader *)((char *)workspace + W.hdr), st, P->opts.sync != 0);
}

int fmm_set_timing(fmm_plan_t P, int on) {
    if (!P) return FMM_ERR_ARG;
    if (on && P->nev_created == 0) {
        for (int i = 0; i < 512; i++) {
            if (cudaEventCreate(&P->ev[i]) != cudaSuccess) return FMM_ERR_CUDA;
            P->nev_created = i + 1;
        }
    }
    P->timing = on != 0;
    P->serial = on == 2;
    return FMM_OK;
}

int fmm_get_stats(fmm_plan_t P, fmm_stats_t *out) {
    if (!P || !out) return FMM_ERR_ARG;
    memset(out, 0, sizeof(*out));
    const Tracer &tr = P->last;
    out->launches = tr.launches;
    if (tr.on && tr.n >= 2) {
        if (cudaEventSynchronize(tr.ev[tr.n - 1]) != cudaSuccess) return FMM_ERR_CUDA;
        for (int k = 0; k + 1 < tr.n; k += 2) {
            float ms = 0;
            if (cudaEventElapsedTime(&ms, tr.ev[k], tr.ev[k + 1]) != cudaSuccess) return FMM_ERR_CUDA;
            int s = tr.stage[k / 2];
            if (s >= 0 && s < FMM_NSTAGES) out->stage_ms[s] += ms;
        }
        out->timed = 1;
    }
    return FMM_OK;
}

int fmm_status(fmm_plan_t P, const void *workspace, void *stream) {
    if (!P) return FMM_ERR_ARG;
    if (!workspace) {  // the scratch array of fmm_eval_static on the current device
        void *ws = nullptr;
        const int rc = fmm::static_workspace_address(&ws);
        if (rc != FMM_OK) return rc;
        workspace = ws;
    }
    return finish(P, (const WsHeader *)((const char *)workspace), (cudaStream_t)stream, true);
}

static int dump_bytes(fmm_plan_t P, int what, int n_eff, size_t *bytes) {
    const size_t rs = P->fp64 ? 8 : 4;
    const int64_t ncell = (int64_t)1 << (3 * P->depth);
    const int p3 = P->p * P->p * P->p;
    int64_t cells = 0;
    for (int l = 0; l <= P->depth; l++) cells += (int64_t)1 << (3 * l);
    switch (what) {
    case FMM_DUMP_COUNTS: *bytes = 16; break;
    case FMM_DUMP_KEYS:
    case FMM_DUMP_ORIGIN:
    case FMM_DUMP_PERM: *bytes = (size_t)n_eff * 4; break;
    case FMM_DUMP_START: *bytes = (size_t)(ncell + 1) * 4; break;
    case FMM_DUMP_POINTS:
    case FMM_DUMP_OUT: *bytes = (size_t)n_eff * 4 * rs; break;
    case FMM_DUMP_WAIT: *bytes = 16; break;
    case FMM_DUMP_PHI:
    case FMM_DUMP_LOCAL: *bytes = (size_t)cells * p3 * rs; break;
    default: return FMM_ERR_ARG;
    }
    return FMM_OK;
}

int fmm_debug_inject(fmm_plan_t P, int what) {
    if (!P) return FMM_ERR_ARG;
    if (what != FMM_INJECT_NONE && what != FMM_INJECT_TC_STALL) return FMM_ERR_ARG;
    if (what == FMM_INJECT_TC_STALL && !P->tc) return FMM_ERR_UNSUPPORTED;
    P->inject = what;
    return FMM_OK;
}

int fmm_debug_size(fmm_plan_t P, int what, const void *workspace, size_t *bytes, void *stream) {
    if (!P || !workspace || !bytes) return FMM_ERR_ARG;
    if (P->last_ws != workspace) return FMM_ERR_STATE;
    WsLayout W = make_layout(P, P->last_n);
    WsHeader h;
    if (cudaMemcpyAsync(&h, (const char *)workspace + W.hdr, sizeof(h), cudaMemcpyDeviceToHost,
                        (cudaStream_t)stream) != cudaSuccess ||
        cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess)
        return FMM_ERR_CUDA;
    return dump_bytes(P, what, h.n_eff, bytes);
}

int fmm_debug_dump(fmm_plan_t P, int what, const void *workspace, void *dst, size_t bytes,
                   void *stream) {
    if (!P || !workspace || !dst) return FMM_ERR_ARG;
    if (P->last_ws != workspace) return FMM_ERR_STATE;
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = P->last_n;
    WsLayout W = make_layout(P, n);
    const char *b = (const char *)workspace;
    WsHeader h;
    if (cudaMemcpyAsync(&h, b + W.hdr, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return FMM_ERR_CUDA;
    size_t need;
    if (dump_bytes(P, what, h.n_eff, &need) || bytes < need) return FMM_ERR_ARG;
    const size_t rs = P->fp64 ? 8 : 4;
    const int p = P->p, p3 = p * p * p;
    auto copy = [&](size_t off, size_t nb) {
        if (nb == 0) return FMM_OK;
        if (cudaMemcpyAsync(dst, b + off, nb, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return FMM_ERR_CUDA;
        return FMM_OK;
    };
    switch (what) {
    case FMM_DUMP_COUNTS: {
        int32_t c[4] = {(int32_t)n, h.n_eff, (int32_t)W.ncell, h.n_coinc};
        memcpy(dst, c, 16);
        return FMM_OK;
    }
    case FMM_DUMP_KEYS: return copy(W.e_key, need);
    case FMM_DUMP_ORIGIN: return copy(W.s_origin, need);
    case FMM_DUMP_PERM: return copy(W.perm, need);
    case FMM_DUMP_START: return copy(W.leaf_start, need);
    case FMM_DUMP_POINTS: return copy(W.s_pt, need);
    case FMM_DUMP_OUT: {
        // results are kept by emitted index: back to sorted order through perm
        std::vector<char> e(need);
        std::vector<int32_t> pm((size_t)h.n_eff);
        if (cudaMemcpyAsync(e.data(), b + W.e_pt, need, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaMemcpyAsync(pm.data(), b + W.perm, pm.size() * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return FMM_ERR_CUDA;
        const size_t row = 4 * rs;
        for (size_t s = 0; s < pm.size(); s++)
            memcpy((char *)dst + s * row, e.data() + (size_t)pm[s] * row, row);
        return FMM_OK;
    }
    case FMM_DUMP_WAIT: {
        int32_t c[4] = {h.wait_site, h.wait_block, h.wait_level, h.wait_iter};
        memcpy(dst, c, 16);
        return FMM_OK;
    }
    case FMM_DUMP_PHI:
    case FMM_DUMP_LOCAL: {
        const bool isphi = what == FMM_DUMP_PHI;
        size_t off = isphi ? W.phi : W.loc;
        int64_t total = isphi ? W.phi_level[P->depth + 1] : W.loc_level[P->depth + 1];
        std::vector<char> raw((size_t)total * rs);
        if (cudaMemcpyAsync(raw.data(), b + off, raw.size(), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return FMM_ERR_CUDA;
        // grid charges are formed on the levels of the upward pass, functionals
        // at the cells that hold charges on the levels of the downward pass
        // (open form: both from level 2); the others are reported as zero
        std::vector<int32_t> start;
        if (!isphi) {
            start.resize((size_t)W.ncell + 1);
            if (cudaMemcpyAsync(start.data(), b + W.leaf_start, start.size() * 4, cudaMemcpyDeviceToHost, st) !=
                    cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess)
                return FMM_ERR_CUDA;
        }
        const int lform = P->periodic ? 0 : 2;
        char *d = (char *)dst;
        size_t o = 0;
        for (int l = 0; l <= P->depth; l++) {
            int S = 1 << l;
            int64_t lvl = isphi ? W.phi_level[l] : W.loc_level[l];
            const int sh = 3 * (P->depth - l);
            for (int cz = 0; cz < S; cz++)
                for (int cy = 0; cy < S; cy++)
                    for (int cx = 0; cx < S; cx++) {
                        int64_t c = isphi ? phi_cell(l, cx, cy, cz) : loc_cell(l, cx, cy, cz);
                        bool formed = l >= lform;  // the open form's upward pass stops at level 2
                        if (!isphi) {
                            const int64_t k = morton_encode(cx, cy, cz);
                            formed = l >= lform && start[(size_t)((k + 1) << sh)] > start[(size_t)(k << sh)];
                        }
                        if (formed)
                            memcpy(d + o, raw.data() + (size_t)(lvl + c * p3) * rs, (size_t)p3 * rs);
                        else
                            memset(d + o, 0, (size_t)p3 * rs);
                        o += (size_t)p3 * rs;
                    }
        }
        return FMM_OK;
    }
    default: return FMM_ERR_ARG;
    }
}

}  // extern "C"

// ---------------------------------------------------------------------------
// batched evaluation
// ---------------------------------------------------------------------------
namespace {

struct Lane {
    cudaStream_t main, near, coarse;
    cudaEvent_t sorted, near_done, fork, coarse_done, join;
};

const int kMaxLanes = 32;
const int kLaneChoices[5] = {2, 4, 8, 16, 32};

// OR of the status words of every system's workspace header
__global__ void k_batch_status(const char *ws, const long long *off, int nsys, int *out) {
    __shared__ int acc;
    if (threadIdx.x == 0) acc = 0;
    __syncthreads();
    int st = 0;
    for (int i = threadIdx.x; i < nsys; i += blockDim.x)
        st |= reinterpret_cast<const WsHeader *>(ws + off[i])->status;
    atomicOr(&acc, st);
    __syncthreads();
    if (threadIdx.x == 0) *out = acc;
}

}  // namespace

struct fmm_batch_s {
    int nsys, p, periodic;
    fmm_opts_t opts;
    std::vector<fmm_plan_t> masters;  // one per distinct depth (owns the tables)
    std::vector<fmm_plan_t> sys;      // per system (shares its master's tables)
    std::vector<int64_t> max_n;
    Lane lane[kMaxLanes];
    int nlanes_made;
    cudaEvent_t fork;
    cudaStream_t cap;            // the graph is captured on and launched from this stream
    cudaEvent_t in_ev, out_ev;   // caller's stream -> cap -> caller's stream
    int *d_status, *h_status;
    long long *d_off;
    // captured graph and what it was captured for
    cudaGraphExec_t gexec;
    int glanes;
    std::vector<int64_t> key;
    int lanes;        // chosen by the autotuner (0: not yet tuned)
    double tune_ms[8];
    int launches;
    bool last_graph;
    // merged form: one launch per call site for all systems (schedule 1: the
    // near-field launches on a forked stream beside the rest, 0: one stream;
    // -1: not yet chosen; merged = false: the systems' sequences do not merge
    // and the stream lanes are used)
    bool merged;
    int schedule;
    cudaStream_t near;
    cudaEvent_t near_fork, near_join;
    char *d_tab;      // per merged launch: the systems' functors and block prefix
    size_t tab_bytes;
    void *d_x;        // cross-system contraction tiles: lists and the systems' table
    size_t x_bytes;
};

namespace {

fmm_plan_t clone_plan(const fmm_plan_s *m, const double *box, int64_t max_n) {
    fmm_plan_s *P = new (std::nothrow) fmm_plan_s(*m);
    if (!P) return nullptr;
    P->id = ++g_plan_counter;
    P->shared = true;
    P->s_near = P->s_coarse = P->s_far = nullptr;
    P->e_sorted = P->e_near = P->e_fork = P->e_coarse = P->e_far = nullptr;
    P->h_hdr = nullptr;
    P->timing = false;
    P->serial = false;
    P->inject = FMM_INJECT_NONE;
    P->nev_created = 0;
    P->max_n = max_n;
    memcpy(P->box, box, sizeof(double) * 4);
    for (int a = 0; a < 3; a++) P->geom.x0[a] = (float)box[a];
    P->geom.Lf = (float)box[3];
    P->geom.L = box[3];
    return P;
}

// One launch of the merged form: the call site's functor type (its launcher),
// its block size and shared memory, and where its functor array and block
// prefix lie in the batch's table.
struct MergedLaunch {
    int tag;
    int near;
    void (*many)(const void *, const int *, int, int, int, size_t, cudaStream_t);
    void (*set_smem)(size_t);
    int threads, total;
    size_t smem;
    size_t ks_off, first_off;
};

// Records every system's launch sequence and merges them: equal tags become
// one launch; the order of the merged launches is a topological order of the
// systems' sequences (ties: first appearance).  Fails (FMM_ERR_UNSUPPORTED)
// where the sequences do not merge: an order that conflicts, or one tag with
// different kernels or launch shapes.  The table (functors, prefixes) is
// uploaded to the device before the call returns.
int record_merged(fmm_batch_t B, const std::vector<int64_t> &n, const std::vector<int64_t> &pofs,
                  const std::vector<size_t> &wofs, const float *pos, const float *q, void *potential,
                  double *energy, void *forces, char *ws, std::vector<MergedLaunch> &out) {
    const int ns = B->nsys;
    if (B->opts.precision == FMM_PREC_FP64) return FMM_ERR_UNSUPPORTED;
    fmm_plan_t M0 = nullptr;  // the tables (shared by every master: same p, kernel and options)
    for (fmm_plan_t m : B->masters)
        if (m && !M0) M0 = m;
    // tensor-core plans: the levels with fewer than 8 coarse cells per axis
    // (l <= 3) of every system run as cross-system tiles, full rows; each
    // system's own contraction takes levels 4 and up
    const int tc_lmin = M0->tc ? (B->periodic ? 1 : 2) : 0;
    const int x_lmax = 3;
    std::vector<std::vector<LaunchRec>> recs(ns);
    const Lane &L = B->lane[0];
    Streams S = {L.main, L.near, L.coarse, L.sorted, L.near_done, L.fork, L.coarse_done, nullptr, nullptr};
    for (int i = 0; i < ns; i++) {
        Tracer tr;
        tr.rec = &recs[i];
        tr.tc_lbig = tc_lmin ? x_lmax + 1 : 0;
        fmm_plan_t P = B->sys[i];
        const int64_t o = pofs[i];
        char *pot = potential ? (char *)potential + o * 4 : nullptr;
        char *frc = forces ? (char *)forces + 3 * o * 4 : nullptr;
        double *en = energy ? energy + i : nullptr;
        int rc = eval_impl<float>(P, n[i], pos + 3 * o, q + o, (float *)pot, en, (float *)frc, ws + wofs[i], S, tr);
        if (rc) return rc;
    }
    if (tc_lmin) {
        // the cross-system tiles, one launch per kernel component, right after
        // the operand split of the first system that has one (merged, that
        // split is every system's)
        std::vector<TcXSys> xs((size_t)M0->ncomp * ns);
        std::vector<int> dep(ns);
        WsLayout W0;
        for (int i = 0; i < ns; i++) {
            WsLayout W = make_layout(B->sys[i], n[i]);
            Ptrs<float> Pi = make_ptrs<float>(W, ws + wofs[i]);
            if (i == 0) W0 = W;
            dep[i] = n[i] > 0 ? B->sys[i]->depth : 0;
            for (int c = 0; c < M0->ncomp; c++)
                xs[(size_t)c * ns + i] = TcXSys{reinterpret_cast<const char *>(Pi.phihi),
                                               reinterpret_cast<const char *>(Pi.philo), Pi.qlev,
                                               Pi.loc + c * W.loc_comp};
        }
        const void *khi[4], *klo[4];
        const float *kb[4];
        for (int c = 0; c < M0->ncomp; c++) {
            khi[c] = M0->khi_map[c];
            klo[c] = M0->klo_map[c];
            kb[c] = (const float *)M0->Kbar_tc + (size_t)c * 343 * tc_padded(M0->geom.p3);
        }
        int *status = &reinterpret_cast<WsHeader *>(ws + wofs[0])->status;
        std::vector<LaunchRec> xr;
        int rc = tc_cross_records(xs, dep, M0->ncomp, tc_lmin, x_lmax, M0->geom.p3, M0->tc_mode, M0->geom.power, khi,
                                  klo, kb, W0, status, &B->d_x, &B->x_bytes, xr);
        if (rc) return rc;
        bool placed = false;
        for (int i = 0; i < ns && !placed; i++)
            for (size_t k = 0; k < recs[i].size() && !placed; k++)
                if (recs[i][k].tag == FMM_TAG(S_SPLIT_TC, 0)) {
                    recs[i].insert(recs[i].begin() + k + 1, xr.begin(), xr.end());
                    placed = true;
                }
    }
    // tags, their first appearance and the edges between consecutive launches
    std::vector<int> tags;
    std::vector<int> first_seen;
    auto index_of = [&](int tag) {
        for (size_t k = 0; k < tags.size(); k++)
            if (tags[k] == tag) return (int)k;
        tags.push_back(tag);
        return (int)tags.size() - 1;
    };
    std::vector<std::vector<int>> seq(ns);
    for (int i = 0; i < ns; i++)
        for (const LaunchRec &r : recs[i]) seq[i].push_back(index_of(r.tag));
    const int nt = (int)tags.size();
    std::vector<std::vector<char>> edge(nt, std::vector<char>(nt, 0));
    std::vector<int> indeg(nt, 0);
    for (int i = 0; i < ns; i++) {
        std::vector<char> seen(nt, 0);
        for (size_t k = 0; k < seq[i].size(); k++) {
            if (seen[seq[i][k]]) return FMM_ERR_UNSUPPORTED;  // one site twice in a system
            seen[seq[i][k]] = 1;
            if (k > 0 && !edge[seq[i][k - 1]][seq[i][k]]) {
                edge[seq[i][k - 1]][seq[i][k]] = 1;
                indeg[seq[i][k]]++;
            }
        }
    }
    std::vector<int> order;
    std::vector<char> done(nt, 0);
    for (int it = 0; it < nt; it++) {
        int pick = -1;
        for (int t = 0; t < nt && pick < 0; t++)
            if (!done[t] && indeg[t] == 0) pick = t;
        if (pick < 0) return FMM_ERR_UNSUPPORTED;  // the orders conflict
        done[pick] = 1;
        order.push_back(pick);
        for (int t = 0; t < nt; t++)
            if (edge[pick][t]) indeg[t]--;
    }
    // per merged launch: the systems' functors and the prefix of their blocks
    std::vector<const LaunchRec *> by(ns);
    std::vector<unsigned char> host;
    auto place = [&](size_t bytes, size_t align) {
        size_t o = (host.size() + align - 1) / align * align;
        host.resize(o + bytes, 0);
        return o;
    };
    out.clear();
    for (int t : order) {
        const LaunchRec *ref = nullptr;
        for (int i = 0; i < ns; i++) {
            by[i] = nullptr;
            for (size_t k = 0; k < recs[i].size(); k++)
                if (seq[i][k] == t) by[i] = &recs[i][k];
            if (!by[i]) continue;
            if (!ref) ref = by[i];
            else if (by[i]->many != ref->many || by[i]->threads != ref->threads || by[i]->smem != ref->smem ||
                     by[i]->ksize != ref->ksize || by[i]->near != ref->near)
                return FMM_ERR_UNSUPPORTED;
        }
        MergedLaunch m;
        m.tag = tags[t];
        m.near = ref->near;
        m.many = ref->many;
        m.set_smem = ref->set_smem;
        m.threads = ref->threads;
        m.smem = ref->smem;
        m.total = 0;
        m.ks_off = m.first_off = 0;
        if (ref->many) {
            const size_t al = ref->kalign < 16 ? 16 : ref->kalign;
            m.ks_off = place(ref->ksize * ns, al < 128 ? 128 : al);
            for (int i = 0; i < ns; i++)
                if (by[i]) memcpy(host.data() + m.ks_off + i * ref->ksize, by[i]->k.data(), ref->ksize);
            m.first_off = place(sizeof(int) * (ns + 1), 16);
            int *first = reinterpret_cast<int *>(host.data() + m.first_off);
            int64_t tot = 0;
            for (int i = 0; i < ns; i++) {
                first[i] = (int)tot;
                tot += by[i] ? by[i]->blocks : 0;
            }
            if (tot > INT32_MAX) return FMM_ERR_UNSUPPORTED;
            first[ns] = (int)tot;
            m.total = (int)tot;
        }
        out.push_back(m);
    }
    if (host.size() > B->tab_bytes) {
        if (B->d_tab) cudaFree(B->d_tab);
        B->d_tab = nullptr;
        B->tab_bytes = 0;
        if (cudaMalloc(&B->d_tab, host.size()) != cudaSuccess) return FMM_ERR_OOM;
        B->tab_bytes = host.size();
    }
    if (!host.empty() && cudaMemcpy(B->d_tab, host.data(), host.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return FMM_ERR_CUDA;
    for (const MergedLaunch &m : out)
        if (m.set_smem && m.smem > 48 * 1024) m.set_smem(m.smem);
    return FMM_OK;
}

// Captures the merged launches: schedule 0 on one stream; schedule 1 with
// the near-field launches on a second stream, each after every launch that
// precedes it in the merged order, joined back at the marker.
int capture_merged(fmm_batch_t B, const std::vector<MergedLaunch> &ml, int schedule, const char *ws,
                   cudaStream_t st, cudaGraphExec_t *out, int *launches) {
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed) != cudaSuccess) return FMM_ERR_CUDA;
    int total = 0;
    // forked: near-field work not yet joined; main_since: main-stream launches
    // issued since the near stream last waited for the main stream.  A near
    // launch waits for every launch before it in the merged order, so the
    // schedule holds for any order the merge gives (a main-stream launch that
    // one system needs before its near field may come after another system's
    // first near launch).
    bool forked = false, main_since = true;
    for (const MergedLaunch &m : ml) {
        if (!m.many) {  // the join marker
            if (forked) {
                cudaEventRecord(B->near_join, B->near);
                cudaStreamWaitEvent(st, B->near_join, 0);
                forked = false;
            }
            continue;
        }
        if (m.total <= 0) continue;
        cudaStream_t s = st;
        if (schedule == 1 && m.near) {
            if (main_since) {
                cudaEventRecord(B->near_fork, st);
                cudaStreamWaitEvent(B->near, B->near_fork, 0);
                main_since = false;
            }
            forked = true;
            s = B->near;
        } else {
            main_since = true;
        }
        m.many(B->d_tab + m.ks_off, reinterpret_cast<const int *>(B->d_tab + m.first_off), B->nsys, m.total,
               m.threads, m.smem, s);
        total++;
    }
    if (forked) {
        cudaEventRecord(B->near_join, B->near);
        cudaStreamWaitEvent(st, B->near_join, 0);
    }
    k_batch_status<<<1, 256, 0, st>>>(ws, B->d_off, B->nsys, B->d_status);
    total++;
    cudaMemcpyAsync(B->h_status, B->d_status, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamEndCapture(st, &graph);
    if (e != cudaSuccess || !graph) return FMM_ERR_CUDA;
    e = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return FMM_ERR_CUDA;
    *launches = total;
    return FMM_OK;
}

int capture_batch(fmm_batch_t B, int lanes, const std::vector<int64_t> &n,
                  const std::vector<int64_t> &pofs, const std::vector<size_t> &wofs, const float *pos,
                  const float *q, void *potential, double *energy, void *forces, char *ws,
                  cudaStream_t st, cudaGraphExec_t *out, int *launches) {
    const size_t rs = B->opts.precision == FMM_PREC_FP64 ? 8 : 4;
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed) != cudaSuccess) return FMM_ERR_CUDA;
    cudaEventRecord(B->fork, st);
    for (int k = 0; k < lanes; k++) cudaStreamWaitEvent(B->lane[k].main, B->fork, 0);
    int rc = FMM_OK, total = 0;
    for (int i = 0; i < B->nsys && rc == FMM_OK; i++) {
        const Lane &L = B->lane[i % lanes];
        Streams S = {L.main, L.near, L.coarse, L.sorted, L.near_done, L.fork, L.coarse_done,
                     nullptr, nullptr};
        Tracer tr;
        tr.st = L.main;
        fmm_plan_t P = B->sys[i];
        const int64_t o = pofs[i];
        char *pot = potential ? (char *)potential + o * rs : nullptr;
        char *frc = forces ? (char *)forces + 3 * o * rs : nullptr;
        double *en = energy ? energy + i : nullptr;
        if (P->fp64)
            rc = eval_impl<double>(P, n[i], pos + 3 * o, q + o, (double *)pot, en, (double *)frc,
                                   ws + wofs[i], S, tr);
        else
            rc = eval_impl<float>(P, n[i], pos + 3 * o, q + o, (float *)pot, en, (float *)frc,
                                  ws + wofs[i], S, tr);
        total += tr.launches;
    }
    for (int k = 0; k < lanes; k++) {
        cudaEventRecord(B->lane[k].join, B->lane[k].main);
        cudaStreamWaitEvent(st, B->lane[k].join, 0);
    }
    k_batch_status<<<1, 256, 0, st>>>(ws, B->d_off, B->nsys, B->d_status);
    total++;
    cudaMemcpyAsync(B->h_status, B->d_status, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamEndCapture(st, &graph);
    if (rc != FMM_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess || !graph) return FMM_ERR_CUDA;
    e = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return FMM_ERR_CUDA;
    *launches = total;
    return FMM_OK;
}

}  // namespace

extern "C" {

int fmm_batch_create(fmm_batch_t *out, int nsys, const double *boxes, const int *depths, int p,
                     int periodic, const fmm_opts_t *opts, const int64_t *max_n) {
    if (!out || nsys <= 0 || !boxes || !depths || !max_n) return FMM_ERR_ARG;
    *out = nullptr;
    fmm_batch_s *B = new (std::nothrow) fmm_batch_s();
    if (!B) return FMM_ERR_OOM;
    B->nsys = nsys;
    B->p = p;
    B->periodic = periodic ? 1 : 0;
    fmm_opts_default(&B->opts);
    if (opts) B->opts = *opts;
    if (B->opts.shift_free) {  // the App. A.2 tables are per plan: single systems only
        delete B;
        return FMM_ERR_UNSUPPORTED;
    }
    B->max_n.assign(max_n, max_n + nsys);
    B->masters.assign(FMM_MAXDEPTH + 1, nullptr);
    int rc = FMM_OK;
    for (int i = 0; i < nsys && rc == FMM_OK; i++) {
        const int d = depths[i];
        if (d < 2 || d > FMM_MAXDEPTH) {
            rc = FMM_ERR_ARG;
            break;
        }
        if (!B->masters[d]) {
            int64_t mx = 0;
            for (int j = 0; j < nsys; j++)
                if (depths[j] == d && max_n[j] > mx) mx = max_n[j];
            rc = fmm_plan_create(&B->masters[d], boxes + 4 * i, d, p, periodic, &B->opts, mx);
            if (rc) break;
        }
        if (!(boxes[4 * i + 3] > 0.0) || max_n[i] < 0) {
            rc = FMM_ERR_ARG;
            break;
        }
        fmm_plan_t c = clone_plan(B->masters[d], boxes + 4 * i, max_n[i]);
        if (!c) {
            rc = FMM_ERR_OOM;
            break;
        }
        B->sys.push_back(c);
    }
    if (rc == FMM_OK) {
        int lo = 0, hi = 0;
        cudaDeviceGetStreamPriorityRange(&lo, &hi);
        for (int k = 0; k < kMaxLanes && rc == FMM_OK; k++) {
            Lane &L = B->lane[k];
            if (cudaStreamCreateWithFlags(&L.main, cudaStreamNonBlocking) != cudaSuccess ||
                cudaStreamCreateWithPriority(&L.near, cudaStreamNonBlocking, lo) != cudaSuccess ||
                cudaStreamCreateWithPriority(&L.coarse, cudaStreamNonBlocking, hi) != cudaSuccess ||
                cudaEventCreateWithFlags(&L.sorted, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&L.near_done, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&L.fork, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&L.coarse_done, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&L.join, cudaEventDisableTiming) != cudaSuccess)
                rc = FMM_ERR_CUDA;
            B->nlanes_made = k + 1;
        }
    }
    if (rc == FMM_OK) {
        if (cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&B->in_ev, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&B->out_ev, cudaEventDisableTiming) != cudaSuccess ||
            cudaMalloc(&B->d_status, sizeof(int)) != cudaSuccess ||
            cudaMallocHost(&B->h_status, sizeof(int)) != cudaSuccess ||
            cudaMalloc(&B->d_off, sizeof(long long) * nsys) != cudaSuccess)
            rc = FMM_ERR_OOM;
    }
    B->merged = true;
    B->schedule = -1;
    if (rc == FMM_OK) {
        int lo = 0, hi = 0;
        cudaDeviceGetStreamPriorityRange(&lo, &hi);
        if (cudaStreamCreateWithPriority(&B->near, cudaStreamNonBlocking, lo) != cudaSuccess ||
            cudaEventCreateWithFlags(&B->near_fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&B->near_join, cudaEventDisableTiming) != cudaSuccess)
            rc = FMM_ERR_CUDA;
    }
    if (rc != FMM_OK) {
        fmm_batch_destroy(B);
        return rc;
    }
    *out = B;
    return FMM_OK;
}

void fmm_batch_destroy(fmm_batch_t B) {
    if (!B) return;
    if (B->gexec) cudaGraphExecDestroy(B->gexec);
    for (fmm_plan_t c : B->sys) delete c;
    for (fmm_plan_t m : B->masters)
        if (m) fmm_plan_destroy(m);
    for (int k = 0; k < B->nlanes_made; k++) {
        Lane &L = B->lane[k];
        if (L.main) cudaStreamDestroy(L.main);
        if (L.near) cudaStreamDestroy(L.near);
        if (L.coarse) cudaStreamDestroy(L.coarse);
        if (L.sorted) cudaEventDestroy(L.sorted);
        if (L.near_done) cudaEventDestroy(L.near_done);
        if (L.fork) cudaEventDestroy(L.fork);
        if (L.coarse_done) cudaEventDestroy(L.coarse_done);
        if (L.join) cudaEventDestroy(L.join);
    }
    if (B->fork) cudaEventDestroy(B->fork);
    if (B->cap) cudaStreamDestroy(B->cap);
    if (B->in_ev) cudaEventDestroy(B->in_ev);
    if (B->out_ev) cudaEventDestroy(B->out_ev);
    if (B->d_status) cudaFree(B->d_status);
    if (B->h_status) cudaFreeHost(B->h_status);
    if (B->d_off) cudaFree(B->d_off);
    if (B->d_tab) cudaFree(B->d_tab);
    if (B->d_x) cudaFree(B->d_x);
    if (B->near) cudaStreamDestroy(B->near);
    if (B->near_fork) cudaEventDestroy(B->near_fork);
    if (B->near_join) cudaEventDestroy(B->near_join);
    delete B;
}

static int batch_layout(fmm_batch_t B, const int64_t *n, std::vector<size_t> &wofs, size_t *total) {
    wofs.resize(B->nsys);
    size_t o = 0;
    for (int i = 0; i < B->nsys; i++) {
        if (n[i] < 0 || n[i] > B->max_n[i]) return FMM_ERR_ARG;
        wofs[i] = o;
        o += align256(make_layout(B->sys[i], n[i]).total);
    }
    *total = o;
    return FMM_OK;
}

int fmm_batch_workspace_size(fmm_batch_t B, const int64_t *n, size_t *bytes) {
    if (!B || !n || !bytes) return FMM_ERR_ARG;
    std::vector<size_t> w;
    return batch_layout(B, n, w, bytes);
}

int fmm_batch_eval(fmm_batch_t B, const int64_t *offsets, const float *pos, const float *q,
                   void *potential, double *energy, void *forces, void *workspace,
                   size_t workspace_bytes, void *stream) {
    if (!B || !offsets) return FMM_ERR_ARG;
    if (!workspace || ((uintptr_t)workspace & 255)) return FMM_ERR_WORKSPACE;
    std::vector<int64_t> n(B->nsys), pofs(B->nsys);
    for (int i = 0; i < B->nsys; i++) {
        pofs[i] = offsets[i];
        n[i] = offsets[i + 1] - offsets[i];
    }
    if (offsets[B->nsys] > 0 && (!pos || !q)) return FMM_ERR_ARG;
    std::vector<size_t> wofs;
    size_t total = 0;
    int rc = batch_layout(B, n.data(), wofs, &total);
    if (rc) return rc;
    if (workspace_bytes < total) return FMM_ERR_WORKSPACE;
    cudaStream_t caller = (cudaStream_t)stream;
    // capture and launch on the batch's own stream (the caller's may be the
    // legacy default stream, which cannot be captured), ordered after the
    // caller's earlier work and before its later work by events
    cudaStream_t st = B->cap;
    cudaEventRecord(B->in_ev, caller);
    cudaStreamWaitEvent(st, B->in_ev, 0);
    char *ws = (char *)workspace;
    // what a captured graph is valid for: pointers and counts
    std::vector<int64_t> key = {(int64_t)(uintptr_t)pos, (int64_t)(uintptr_t)q,
                                (int64_t)(uintptr_t)potential, (int64_t)(uintptr_t)energy,
                                (int64_t)(uintptr_t)forces, (int64_t)(uintptr_t)workspace};
    key.insert(key.end(), n.begin(), n.end());
    cudaGetLastError();
    B->last_graph = true;
    std::vector<MergedLaunch> ml;
    if (!B->gexec || key != B->key || (!B->merged && B->lanes && B->glanes != B->lanes)) {
        // the table and offsets are rewritten: nothing of an earlier call may still read them
        if (cudaStreamSynchronize(st) != cudaSuccess) return FMM_ERR_CUDA;
        std::vector<long long> off(B->nsys);
        for (int i = 0; i < B->nsys; i++) off[i] = (long long)wofs[i];
        if (cudaMemcpy(B->d_off, off.data(), sizeof(long long) * B->nsys, cudaMemcpyHostToDevice) !=
            cudaSuccess)
            return FMM_ERR_CUDA;
        if (B->gexec) {
            cudaGraphExecDestroy(B->gexec);
            B->gexec = nullptr;
        }
        // the merged form where the systems' sequences merge, else stream lanes
        rc = B->merged ? record_merged(B, n, pofs, wofs, pos, q, potential, energy, forces, ws, ml)
                       : FMM_ERR_UNSUPPORTED;
        if (rc != FMM_OK && rc != FMM_ERR_UNSUPPORTED) return rc;
        B->merged = rc == FMM_OK;
        // the offsets and tables above went up by cudaMemcpy from pageable
        // memory, which may return before the transfer lands, and the batch's
        // stream is not ordered after it: wait for it before any launch reads them
        if (cudaDeviceSynchronize() != cudaSuccess) return FMM_ERR_CUDA;
    }
    if (!B->gexec && B->merged) {
        if (B->schedule < 0) {
            // autotune the schedule: time each candidate's graph
            cudaEvent_t a, b;
            cudaEventCreate(&a);
            cudaEventCreate(&b);
            double best = 1e30;
            int best_s = 0;
            for (int c = 0; c < 2 && rc == FMM_OK; c++) {
                cudaGraphExec_t ex = nullptr;
                int launches = 0;
                rc = capture_merged(B, ml, c, ws, st, &ex, &launches);
                if (rc) break;
                cudaGraphLaunch(ex, st);  // warm-up
                cudaEventRecord(a, st);
                for (int r = 0; r < 3; r++) cudaGraphLaunch(ex, st);
                cudaEventRecord(b, st);
                cudaEventSynchronize(b);
                float ms = 0;
                cudaEventElapsedTime(&ms, a, b);
                B->tune_ms[5 + c] = ms / 3.0;
                if (ms < best) {
                    best = ms;
                    best_s = c;
                }
                cudaGraphExecDestroy(ex);
            }
            cudaEventDestroy(a);
            cudaEventDestroy(b);
            if (rc) return rc;
            B->schedule = best_s;
        }
        rc = capture_merged(B, ml, B->schedule, ws, st, &B->gexec, &B->launches);
        if (rc) return rc;
        B->key = key;
    }
    if (!B->gexec) {
        if (!B->lanes) {
            // autotune the number of stream lanes: time each candidate's graph
            cudaEvent_t a, b;
            cudaEventCreate(&a);
            cudaEventCreate(&b);
            double best = 1e30;
            int best_l = 2;
            for (int c = 0; c < 5; c++) {
                const int l = kLaneChoices[c] < B->nsys ? kLaneChoices[c] : B->nsys;
                cudaGraphExec_t ex = nullptr;
                int launches = 0;
                rc = capture_batch(B, l, n, pofs, wofs, pos, q, potential, energy, forces, ws, st, &ex,
                                   &launches);
                if (rc) break;
                cudaGraphLaunch(ex, st);  // warm-up
                cudaEventRecord(a, st);
                for (int r = 0; r < 3; r++) cudaGraphLaunch(ex, st);
                cudaEventRecord(b, st);
                cudaEventSynchronize(b);
                float ms = 0;
                cudaEventElapsedTime(&ms, a, b);
                B->tune_ms[c] = ms / 3.0;
                if (ms < best) {
                    best = ms;
                    best_l = l;
                }
                cudaGraphExecDestroy(ex);
                if (kLaneChoices[c] >= B->nsys) break;
            }
            cudaEventDestroy(a);
            cudaEventDestroy(b);
            if (rc) return rc;
            B->lanes = best_l;
        }
        rc = capture_batch(B, B->lanes, n, pofs, wofs, pos, q, potential, energy, forces, ws, st,
                           &B->gexec, &B->launches);
        if (rc) return rc;
        B->glanes = B->lanes;
        B->key = key;
    }
    if (cudaGraphLaunch(B->gexec, st) != cudaSuccess) return FMM_ERR_CUDA;
    cudaEventRecord(B->out_ev, st);
    cudaStreamWaitEvent(caller, B->out_ev, 0);
    if (cudaGetLastError() != cudaSuccess) return FMM_ERR_CUDA;
    if (!B->opts.sync) return FMM_OK;
    if (cudaStreamSynchronize(st) != cudaSuccess) return FMM_ERR_CUDA;
    return status_to_error(*B->h_status);
}

int fmm_batch_get_stats(fmm_batch_t B, fmm_batch_stats_t *out) {
    if (!B || !out) return FMM_ERR_ARG;
    memset(out, 0, sizeof(*out));
    out->launches = B->launches;
    out->lanes = B->merged ? 0 : B->lanes;
    out->graph = B->last_graph ? 1 : 0;
    for (int c = 0; c < 8; c++) out->tune_ms[c] = B->tune_ms[c];
    out->merged = B->merged ? 1 : 0;
    out->schedule = B->merged ? B->schedule : -1;
    return FMM_OK;
}

int fmm_batch_set_schedule(fmm_batch_t B, int schedule) {
    if (!B || schedule < -1 || schedule > 1) return FMM_ERR_ARG;
    B->schedule = schedule;
    B->key.clear();  // the next call records and captures again
    return FMM_OK;
}

}  // extern "C"

/*
 * FP64 CPU oracle of the replacement-based fast multipole method of
 * Y. Kajima, "Notes on the Fast Multipole Method" (arXiv:2212.13080).
 *
 * TEST INFRASTRUCTURE ONLY.  The test suite, the smoke check and the CPU
 * baseline leg of the benchmark are the only callers.  The product library
 * never links, loads or calls this file, and this file shares no source,
 * header, table or constant generator with the CUDA library.
 *
 * Every routine is a plain, slow transcription of the paper's definitions in
 * double precision, in the order the paper gives them.  No blocking, fusion or
 * reordering beyond what a definition states; loops over independent outputs
 * may run on several OpenMP threads, which does not change any output's
 * summation order.
 *
 * Coordinates.  The box [x0, x0+L)^3 is mapped onto the unit cube: the
 * canonical single-precision map u = fl32(fl32(x - x0) / fl32(L)) is the one
 * place where single precision is used, so that leaf membership (integer work)
 * is decided on exactly the same numbers as the GPU path.  Everything after it
 * runs in FP64 on the widened values.  Potentials and forces come out in
 * unit-cube units; the Python driver scales them by 1/L and 1/L^2.
 *
 * Index conventions.
 *   grid vector of a cell:   index (k*n + j)*n + i  for node (i, j, k), x fastest
 *   cell of level l:         natural index (cz*S + cy)*S + cx, S = 2^l
 *   leaf key:                Morton interleave, bit b of cx -> 3b, cy -> 3b+1,
 *                            cz -> 3b+2
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXN 12

#define ORC_ERR_OUT_OF_BOX 1
#define ORC_ERR_NONFINITE 2

/* ------------------------------------------------------------------------ */
/* §2.1.1-§2.1.2: n-division points and the Lagrange basis                  */
/* ------------------------------------------------------------------------ */

/* §2.1.2: the n-division points of a segment are equally spaced and include
 * both end points; on the unit segment they are a_i = i/(n-1).  §4.1 (the
 * "reduced" arrangement) moves them toward the centre of the cell: their
 * spacing is multiplied by a factor s <= 1, a_i = 1/2 + s (i/(n-1) - 1/2). */
static double g_grid_scale = 1.0;
void orc_set_grid_scale(double s) { g_grid_scale = s; }
static double tau(int n, int i) { return 0.5 + g_grid_scale * ((double)i / (double)(n - 1) - 0.5); }

/* §2.1.1, eq. (Lag1): g_i(x) = prod_{k!=i} (x - a_k) / prod_{k!=i} (a_i - a_k). */
void orc_lagrange(int n, double x, double *g)
{
    for (int i = 0; i < n; i++) {
        double num = 1.0, den = 1.0;
        for (int k = 0; k < n; k++) {
            if (k == i) continue;
            num *= x - tau(n, k);
            den *= tau(n, i) - tau(n, k);
        }
        g[i] = num / den;
    }
}

/* d g_i / dx of eq. (Lag1), by the product rule.  The far-field force at the
 * end of §2.2 uses v'_a = -q d/da g_{ijk}. */
void orc_lagrange_deriv(int n, double x, double *dg)
{
    for (int i = 0; i < n; i++) {
        double den = 1.0;
        for (int k = 0; k < n; k++)
            if (k != i) den *= tau(n, i) - tau(n, k);
        double sum = 0.0;
        for (int m = 0; m < n; m++) {
            if (m == i) continue;
            double prod = 1.0;
            for (int k = 0; k < n; k++)
                if (k != i && k != m) prod *= x - tau(n, k);
            sum += prod;
        }
        dg[i] = sum / den;
    }
}

/* §2.1.6, eq. (trans): the shift from a child segment to its parent has
 * (j,i) entry g~_j(a_i): the parent's basis evaluated at the child's nodes.
 * In parent-local coordinates the child h (0 = lower half, 1 = upper half)
 * has nodes (h + a_i)/2.  G[J*n + i]. */
void orc_shift_matrix(int n, int h, double *G)
{
    double g[ORC_MAXN];
    for (int i = 0; i < n; i++) {
        orc_lagrange(n, 0.5 * ((double)h + tau(n, i)), g);
        for (int J = 0; J < n; J++) G[J * n + i] = g[J];
    }
}

/* The function F of the bilinear forms.  §2.1.7 takes F(P, P~) = 1/|P - P~|;
 * the discussion of other kernels (§4.1) notes that the same replacement
 * gives the forces directly with F = (x - x~)/|P - P~|^3 (and its y, z
 * components) instead of differentiating the replaced charges' weights.
 * g_kernel: 0 = 1/r, 1..3 = the x, y, z component of r/|r|^3.  At level l,
 * unit-cell distances are 2^l times unit-box distances, so the forms scale
 * by 2^l (potential) or 4^l (force components). */
static int g_kernel = 0;
void orc_set_kernel(int c) { g_kernel = c; }
/* The same remark names 1/|P - P~|^2 as another function the replacement
 * applies to.  g_power = 1: F = 1/r (default); g_power = 2: F = 1/r^2, whose
 * force components are 2 (x - x~)/r^4.  Forms scale by 2^(l g_power) and
 * 2^(l (g_power + 1)) at level l. */
static int g_power = 1;
void orc_set_power(int k) { g_power = k; }
static double kernel_value(double dx, double dy, double dz)
{
    double r2 = dx * dx + dy * dy + dz * dz, r = sqrt(r2);
    if (g_power == 2) {
        if (g_kernel == 0) return 1.0 / r2;
        double d = g_kernel == 1 ? dx : g_kernel == 2 ? dy : dz;
        return 2.0 * d / (r2 * r2);
    }
    if (g_kernel == 0) return 1.0 / r;
    double d = g_kernel == 1 ? dx : g_kernel == 2 ? dy : dz;
    return d / (r2 * r);
}
static double level_scale(int l) { return ldexp(1.0, g_kernel == 0 ? g_power * l : (g_power + 1) * l); }

/* §2.1.7, eqs. (newer), (bilinear): F(P(a), P(a~)) = 1/|a - a~| between the
 * n-division points a of the unit cell at the origin and a~ of the unit cell
 * displaced by the integer vector o (or the force component selected by
 * orc_set_kernel).  K[a*n^3 + b]. */
void orc_m2l_kernel(int n, int ox, int oy, int oz, double *K)
{
    int n3 = n * n * n;
    for (int a = 0; a < n3; a++) {
        double ax = tau(n, a % n), ay = tau(n, (a / n) % n), az = tau(n, a / (n * n));
        for (int b = 0; b < n3; b++) {
            double bx = ox + tau(n, b % n), by = oy + tau(n, (b / n) % n),
                   bz = oz + tau(n, b / (n * n));
            K[(int64_t)a * n3 + b] = kernel_value(ax - bx, ay - by, az - bz);
        }
    }
}

/* ------------------------------------------------------------------------ */
/* §4.2: periodic boundary by Ewald summation (unit cubic box, tin-foil)     */
/* ------------------------------------------------------------------------ */

/* Ewald splitting constants for the unit box: real-space images |m|_inf <= 5
 * and reciprocal vectors |h|_inf <= 6 with alpha = 2.5 leave truncation terms
 * below 1e-40 and 1e-16 for every r in [-1,1]^3. */
#define EW_ALPHA 2.5
#define EW_RMAX 5
#define EW_KMAX 6

/* Lattice kernel of the level-0 cell (the box) with all of its periodic
 * images that are not among its 26 nearest:
 *   psi(r) = sum_{m not in {-1,0,1}^3} 1/|r + m|   (Ewald-regularised),
 * written as the Ewald pair potential minus the 27 nearest image terms.  The
 * real-space terms of the nearest images become -erf(alpha s)/s, whose limit
 * at s = 0 is -2 alpha/sqrt(pi).  The neutralising-background constant
 * -pi/alpha^2 is kept; it cancels for neutral systems because replacement
 * conserves the total charge (eq. (Lag2) with j = 0). */
double orc_lattice_psi(double rx, double ry, double rz)
{
    const double al = EW_ALPHA;
    double s = 0.0;
    for (int mz = -EW_RMAX; mz <= EW_RMAX; mz++)
        for (int my = -EW_RMAX; my <= EW_RMAX; my++)
            for (int mx = -EW_RMAX; mx <= EW_RMAX; mx++) {
                double dx = rx + mx, dy = ry + my, dz = rz + mz;
                double d = sqrt(dx * dx + dy * dy + dz * dz);
                int nearest = (abs(mx) <= 1 && abs(my) <= 1 && abs(mz) <= 1);
                if (nearest) {
                    if (d == 0.0) s -= 2.0 * al / sqrt(M_PI);
                    else s -= erf(al * d) / d;
                } else {
                    s += erfc(al * d) / d;
                }
            }
    for (int hz = -EW_KMAX; hz <= EW_KMAX; hz++)
        for (int hy = -EW_KMAX; hy <= EW_KMAX; hy++)
            for (int hx = -EW_KMAX; hx <= EW_KMAX; hx++) {
                if (hx == 0 && hy == 0 && hz == 0) continue;
                double h2 = (double)(hx * hx + hy * hy + hz * hz);
                double A = exp(-M_PI * M_PI * h2 / (al * al)) / h2;
                s += A / M_PI * cos(2.0 * M_PI * (hx * rx + hy * ry + hz * rz));
            }
    s -= M_PI / (al * al);
    return s;
}

/* Gradient of psi: term by term, d/dr [erfc(al d)/d] and d/dr [-erf(al d)/d]
 * along r + m, and -2 A h sin(2 pi h.r) for the reciprocal terms; the
 * nearest-image term is even and smooth at d = 0, where its gradient is 0. */
void orc_lattice_grad(double rx, double ry, double rz, double *g)
{
    const double al = EW_ALPHA;
    g[0] = g[1] = g[2] = 0.0;
    for (int mz = -EW_RMAX; mz <= EW_RMAX; mz++)
        for (int my = -EW_RMAX; my <= EW_RMAX; my++)
            for (int mx = -EW_RMAX; mx <= EW_RMAX; mx++) {
                double dx = rx + mx, dy = ry + my, dz = rz + mz;
                double d = sqrt(dx * dx + dy * dy + dz * dz);
                int nearest = (abs(mx) <= 1 && abs(my) <= 1 && abs(mz) <= 1);
                if (d == 0.0) continue;
                double gauss = 2.0 * al / sqrt(M_PI) * exp(-al * al * d * d) / d;
                double dd = nearest ? -gauss + erf(al * d) / (d * d)      /* d/dd of -erf/d */
                                    : -gauss - erfc(al * d) / (d * d);    /* d/dd of erfc/d */
                g[0] += dd * dx / d;
                g[1] += dd * dy / d;
                g[2] += dd * dz / d;
            }
    for (int hz = -EW_KMAX; hz <= EW_KMAX; hz++)
        for (int hy = -EW_KMAX; hy <= EW_KMAX; hy++)
            for (int hx = -EW_KMAX; hx <= EW_KMAX; hx++) {
                if (hx == 0 && hy == 0 && hz == 0) continue;
                double h2 = (double)(hx * hx + hy * hy + hz * hz);
                double A = exp(-M_PI * M_PI * h2 / (al * al)) / h2;
                double sn = sin(2.0 * M_PI * (hx * rx + hy * ry + hz * rz));
                g[0] -= 2.0 * A * hx * sn;
                g[1] -= 2.0 * A * hy * sn;
                g[2] -= 2.0 * A * hz * sn;
            }
}

/* K_lat[a*n^3 + b] = psi(a - b) for the n-division points of the unit box
 * (force component c of orc_set_kernel: -d psi / d r_c at a - b).
 * psi depends on a - b only, which takes (2n-1)^3 distinct values; each is
 * evaluated once. */
void orc_lattice_kernel(int n, double *K)
{
    int n3 = n * n * n, m = 2 * n - 1;
    double *tab = (double *)malloc(sizeof(double) * (size_t)m * m * m);
#pragma omp parallel for schedule(dynamic, 1)
    for (int e = 0; e < m * m * m; e++) {
        int dx = e % m - (n - 1), dy = (e / m) % m - (n - 1), dz = e / (m * m) - (n - 1);
        double rx = tau(n, dx > 0 ? dx : 0) - tau(n, dx < 0 ? -dx : 0);
        double ry = tau(n, dy > 0 ? dy : 0) - tau(n, dy < 0 ? -dy : 0);
        double rz = tau(n, dz > 0 ? dz : 0) - tau(n, dz < 0 ? -dz : 0);
        if (g_kernel == 0) {
            tab[e] = orc_lattice_psi(rx, ry, rz);
        } else {
            double g[3];
            orc_lattice_grad(rx, ry, rz, g);
            tab[e] = -g[g_kernel - 1];
        }
    }
    for (int a = 0; a < n3; a++)
        for (int b = 0; b < n3; b++) {
            int dx = a % n - b % n + n - 1;
            int dy = (a / n) % n - (b / n) % n + n - 1;
            int dz = a / (n * n) - b / (n * n) + n - 1;
            K[(int64_t)a * n3 + b] = tab[(dz * m + dy) * m + dx];
        }
    free(tab);
}

/* Plain Ewald sum (tin-foil boundary, neutralising background) of the
 * potential and field at particles tgt[] of a periodic unit box; the truth for
 * the periodic form of §4.2.  x is 3N unit-cube coordinates.  phi[t] is the
 * potential per unit charge at particle tgt[t] from all other charges and all
 * images (its own images included); F[3t..] = q_i * field. */
void orc_ewald_direct(int64_t N, const double *x, const double *q, int64_t nt,
                      const int64_t *tgt, double *phi, double *F)
{
    const double al = EW_ALPHA;
    const int RM = 4; /* after minimum-image wrap, |r+m| >= 4.1 beyond this */
    double qtot = 0.0;
    for (int64_t j = 0; j < N; j++) qtot += q[j];
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t t = 0; t < nt; t++) {
        int64_t i = tgt[t];
        double p = 0.0, fx = 0.0, fy = 0.0, fz = 0.0;
        for (int64_t j = 0; j < N; j++) {
            double r0[3];
            for (int a = 0; a < 3; a++) {
                double d = x[3 * i + a] - x[3 * j + a];
                r0[a] = d - floor(d + 0.5);
            }
            for (int mz = -RM; mz <= RM; mz++)
                for (int my = -RM; my <= RM; my++)
                    for (int mx = -RM; mx <= RM; mx++) {
                        double dx = r0[0] + mx, dy = r0[1] + my, dz = r0[2] + mz;
                        double s2 = dx * dx + dy * dy + dz * dz;
                        if (j == i && mx == 0 && my == 0 && mz == 0) continue;
                        if (s2 == 0.0) continue;
                        double s = sqrt(s2);
                        double ec = erfc(al * s) / s;
                        p += q[j] * ec;
                        double g = (ec + 2.0 * al / sqrt(M_PI) * exp(-al * al * s2)) / s2;
                        fx += q[j] * g * dx;
                        fy += q[j] * g * dy;
                        fz += q[j] * g * dz;
                    }
        }
        for (int hz = -EW_KMAX; hz <= EW_KMAX; hz++)
            for (int hy = -EW_KMAX; hy <= EW_KMAX; hy++)
                for (int hx = -EW_KMAX; hx <= EW_KMAX; hx++) {
                    if (hx == 0 && hy == 0 && hz == 0) continue;
                    double h2 = (double)(hx * hx + hy * hy + hz * hz);
                    double A = exp(-M_PI * M_PI * h2 / (al * al)) / h2;
                    double c = 0.0, sn = 0.0;
                    for (int64_t j = 0; j < N; j++) {
                        double arg = 2.0 * M_PI * (hx * (x[3 * i] - x[3 * j]) +
                                                   hy * (x[3 * i + 1] - x[3 * j + 1]) +
                                                   hz * (x[3 * i + 2] - x[3 * j + 2]));
                        c += q[j] * cos(arg);
                        sn += q[j] * sin(arg);
                    }
                    p += A / M_PI * c;
                    fx += 2.0 * A * hx * sn;
                    fy += 2.0 * A * hy * sn;
                    fz += 2.0 * A * hz * sn;
                }
        p -= 2.0 * al / sqrt(M_PI) * q[i];
        p -= M_PI / (al * al) * qtot;
        phi[t] = p;
        F[3 * t] = q[i] * fx;
        F[3 * t + 1] = q[i] * fy;
        F[3 * t + 2] = q[i] * fz;
    }
}

/* Plain O(N^2) Coulomb sum (or the 1/r^2 sum, orc_set_power(2)), open boundary:
 * phi_i = sum_{j != i} q_j/|x_i - x_j|
 * and F_i = q_i sum_{j != i} q_j (x_i - x_j)/|x_i - x_j|^3, at particles tgt[].
 * Coincident pairs are skipped. */
void orc_direct_open(int64_t N, const double *x, const double *q, int64_t nt,
                     const int64_t *tgt, double *phi, double *F)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < nt; t++) {
        int64_t i = tgt[t];
        double p = 0.0, fx = 0.0, fy = 0.0, fz = 0.0;
        for (int64_t j = 0; j < N; j++) {
            if (j == i) continue;
            double dx = x[3 * i] - x[3 * j], dy = x[3 * i + 1] - x[3 * j + 1],
                   dz = x[3 * i + 2] - x[3 * j + 2];
            double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 == 0.0) continue;
            double r = sqrt(r2);
            /* 1/r, or 1/r^2 (orc_set_power(2)) with force 2 q q' r/r^4 */
            p += g_power == 2 ? q[j] / r2 : q[j] / r;
            double c = g_power == 2 ? 2.0 * q[j] / (r2 * r2) : q[j] / (r2 * r);
            fx += c * dx;
            fy += c * dy;
            fz += c * dz;
        }
        phi[t] = p;
        F[3 * t] = q[i] * fx;
        F[3 * t + 1] = q[i] * fy;
        F[3 * t + 2] = q[i] * fz;
    }
}

/* ------------------------------------------------------------------------ */
/* §2.2 step 1: divide the simulation box                                    */
/* ------------------------------------------------------------------------ */

static uint32_t morton3(int x, int y, int z, int depth)
{
    uint32_t k = 0;
    for (int b = 0; b < depth; b++) {
        k |= (uint32_t)((x >> b) & 1) << (3 * b);
        k |= (uint32_t)((y >> b) & 1) << (3 * b + 1);
        k |= (uint32_t)((z >> b) & 1) << (3 * b + 2);
    }
    return k;
}

static void demorton3(uint32_t k, int depth, int *x, int *y, int *z)
{
    *x = *y = *z = 0;
    for (int b = 0; b < depth; b++) {
        *x |= (int)((k >> (3 * b)) & 1u) << b;
        *y |= (int)((k >> (3 * b + 1)) & 1u) << b;
        *z |= (int)((k >> (3 * b + 2)) & 1u) << b;
    }
}

uint32_t orc_morton(int x, int y, int z, int depth) { return morton3(x, y, z, depth); }

/* Step 1 of §2.2 divides the box into 8^depth finest cells.  The map from a
 * position to its finest cell is not spelled out in the paper; it is taken
 * here as the canonical single-precision map
 *   u = fl32(fl32(x - x0) / fl32(L)),  c = min(floor(u 2^depth), 2^depth - 1),
 *   t = u 2^depth - c   (exact: 2^depth is a power of two),
 * with u wrapped into [0,1) in the periodic form (§4.2) and rejected outside
 * [0,1) in the open form.  A particle exactly on a plane belongs to the upper
 * cell.  Returns a bit set of ORC_ERR_* flags. */
int orc_bin(int64_t N, const float *pos, const double *box, int depth, int periodic,
            float *u_out, float *t_out, int32_t *cell_out, uint32_t *key_out)
{
    const float x0[3] = {(float)box[0], (float)box[1], (float)box[2]};
    const float Lf = (float)box[3];
    const int S = 1 << depth;
    const float Sf = (float)S;
    int err = 0;
    for (int64_t i = 0; i < N; i++) {
        int c[3];
        for (int a = 0; a < 3; a++) {
            float d = pos[3 * i + a] - x0[a];
            float u = d / Lf;
            if (!isfinite(u)) {
                err |= ORC_ERR_NONFINITE;
                u = 0.0f;
            }
            if (periodic) {
                u = u - floorf(u);
                if (u >= 1.0f) u = 0.0f;
            } else if (!(u >= 0.0f && u < 1.0f)) {
                err |= ORC_ERR_OUT_OF_BOX;
                u = 0.0f;
            }
            float v = u * Sf;
            int ci = (int)floorf(v);
            if (ci > S - 1) ci = S - 1;
            u_out[3 * i + a] = u;
            t_out[3 * i + a] = v - (float)ci;
            cell_out[3 * i + a] = ci;
            c[a] = ci;
        }
        key_out[i] = morton3(c[0], c[1], c[2], depth);
    }
    return err;
}

/* ------------------------------------------------------------------------ */
/* §2.3: split of particles that lie closer than d to a plane of the finest  */
/* cells (continuous form); §4.2 adds the walls of the periodic box.         */
/* ------------------------------------------------------------------------ */

/* One axis of the split of one particle: up to n+1 entries of
 * (cell, local coordinate, weight, d weight / du). */
typedef struct {
    int m;
    int cell[ORC_MAXN + 1];
    double t[ORC_MAXN + 1];
    double w[ORC_MAXN + 1];
    double dw[ORC_MAXN + 1];
} axis_split;

/* §2.3: a particle within distance d (< d, strict) of a plane is replaced by n
 * charges on a segment of length 2d perpendicular to the plane, centred on
 * it, with weights given by the one-dimensional replacement (§2.1.3) onto the
 * segment's n-division points.  dt = d / (leaf width) in leaf units.  Planes
 * are the interior planes of the finest cells; the periodic form also splits
 * at the box walls, identifying the points outside with their images inside
 * (§4.2).  Odd n: the middle point lies on the plane and is divided into two
 * half charges, one in each adjacent cell (first option of §2.3). */
static void split_axis(int n, int depth, int periodic, int continuous, float dtf, int c,
                       float t, axis_split *s)
{
    const int S = 1 << depth;
    const float hi = 1.0f - dtf;
    int lower = continuous && (periodic || c > 0) && t < dtf;
    int upper = continuous && (periodic || c < S - 1) && t > hi;
    if (!lower && !upper) {
        s->m = 1;
        s->cell[0] = c;
        s->t[0] = (double)t;
        s->w[0] = 1.0;
        s->dw[0] = 0.0;
        return;
    }
    const double dt = (double)dtf;
    int cl, cu;        /* cells below and above the plane */
    double sigma;      /* signed distance from the plane in units of d */
    if (lower) {
        cl = c - 1;
        cu = c;
        sigma = (double)t / dt;
    } else {
        cl = c;
        cu = c + 1;
        sigma = ((double)t - 1.0) / dt;
    }
    if (periodic) {
        cl = (cl + S) % S;
        cu = cu % S;
    }
    double g[ORC_MAXN], dg[ORC_MAXN];
    double x = 0.5 * (sigma + 1.0); /* segment nodes -1 + 2k/(n-1) <-> tau_k */
    orc_lagrange(n, x, g);
    orc_lagrange_deriv(n, x, dg);
    /* d x / d u = (1/2) * (1/dt) * 2^depth */
    const double dxdu = 0.5 / dt * (double)S;
    int m = 0;
    for (int k = 0; k < n; k++) {
        double sk = -1.0 + 2.0 * (double)k / (double)(n - 1);
        if (2 * k == n - 1) {
            s->cell[m] = cl; s->t[m] = 1.0; s->w[m] = 0.5 * g[k]; s->dw[m] = 0.5 * dg[k] * dxdu; m++;
            s->cell[m] = cu; s->t[m] = 0.0; s->w[m] = 0.5 * g[k]; s->dw[m] = 0.5 * dg[k] * dxdu; m++;
        } else if (2 * k < n - 1) {
            s->cell[m] = cl; s->t[m] = 1.0 + sk * dt; s->w[m] = g[k]; s->dw[m] = dg[k] * dxdu; m++;
        } else {
            s->cell[m] = cu; s->t[m] = sk * dt; s->w[m] = g[k]; s->dw[m] = dg[k] * dxdu; m++;
        }
    }
    s->m = m;
}

/* Number of charges each particle becomes: the product over the three axes
 * (1, n, or n+1 for odd n); the paper's n, n^2, n^3 cases of §2.3.
 * axes[3i+a] = 1 where particle i is split along axis a. */
void orc_split_count(int64_t N, const float *t, const int32_t *cell, int n, int depth,
                     int periodic, int continuous, float dtf, int32_t *count, int8_t *axes)
{
    for (int64_t i = 0; i < N; i++) {
        int c = 1;
        for (int a = 0; a < 3; a++) {
            axis_split s;
            split_axis(n, depth, periodic, continuous, dtf, cell[3 * i + a], t[3 * i + a], &s);
            c *= s.m;
            axes[3 * i + a] = (int8_t)(s.m > 1);
        }
        count[i] = c;
    }
}

/* Emits the charges of every particle, particle after particle, each as the
 * tensor product of its three axes with x fastest (§2.3: n^2 and n^3 near
 * edges and corners).  offset[i] = first output slot of particle i. */
void orc_split_emit(int64_t N, const float *t, const int32_t *cell, const float *q, int n,
                    int depth, int periodic, int continuous, float dtf, const int64_t *offset,
                    double *pt_t, int32_t *pt_cell, uint32_t *pt_key, double *pt_q,
                    double *pt_w, double *pt_dw, int64_t *pt_origin)
{
    for (int64_t i = 0; i < N; i++) {
        axis_split s[3];
        for (int a = 0; a < 3; a++)
            split_axis(n, depth, periodic, continuous, dtf, cell[3 * i + a], t[3 * i + a], &s[a]);
        int64_t o = offset[i];
        for (int kz = 0; kz < s[2].m; kz++)
            for (int ky = 0; ky < s[1].m; ky++)
                for (int kx = 0; kx < s[0].m; kx++) {
                    double W = s[0].w[kx] * s[1].w[ky] * s[2].w[kz];
                    pt_t[3 * o] = s[0].t[kx];
                    pt_t[3 * o + 1] = s[1].t[ky];
                    pt_t[3 * o + 2] = s[2].t[kz];
                    pt_cell[3 * o] = s[0].cell[kx];
                    pt_cell[3 * o + 1] = s[1].cell[ky];
                    pt_cell[3 * o + 2] = s[2].cell[kz];
                    pt_key[o] = morton3(s[0].cell[kx], s[1].cell[ky], s[2].cell[kz], depth);
                    pt_w[o] = W;
                    pt_q[o] = (double)q[i] * W;
                    pt_dw[3 * o] = s[0].dw[kx] * s[1].w[ky] * s[2].w[kz];
                    pt_dw[3 * o + 1] = s[0].w[kx] * s[1].dw[ky] * s[2].w[kz];
                    pt_dw[3 * o + 2] = s[0].w[kx] * s[1].w[ky] * s[2].dw[kz];
                    pt_origin[o] = i;
                    o++;
                }
    }
}

/* Stable counting sort of the charges by finest-cell key: perm[s] = emitted
 * index of sorted slot s, start[key] = first slot of the cell.  Ties keep
 * their emitted order. */
void orc_sort(int64_t npts, const uint32_t *key, int depth, int64_t *perm, int64_t *start)
{
    int64_t ncell = (int64_t)1 << (3 * depth);
    for (int64_t c = 0; c <= ncell; c++) start[c] = 0;
    for (int64_t e = 0; e < npts; e++) start[key[e] + 1]++;
    for (int64_t c = 0; c < ncell; c++) start[c + 1] += start[c];
    int64_t *cur = (int64_t *)malloc(sizeof(int64_t) * (size_t)ncell);
    for (int64_t c = 0; c < ncell; c++) cur[c] = start[c];
    for (int64_t e = 0; e < npts; e++) perm[cur[key[e]]++] = e;
    free(cur);
}

/* ------------------------------------------------------------------------ */
/* §2.2 step 2: upward pass (replacement at the leaves, then shift upward)   */
/* ------------------------------------------------------------------------ */

static int64_t level_offset(int n, int l)
{
    int64_t n3 = (int64_t)n * n * n, cells = 0;
    for (int k = 0; k < l; k++) cells += (int64_t)1 << (3 * k);
    return cells * n3;
}

int64_t orc_level_offset(int n, int l) { return level_offset(n, l); }

/* §2.1.5, eq. (ex66): replacement of the charges of each finest cell with
 * respect to that cell, Phi[i,j,k] = sum_l q_l g_i(x_l) g_j(y_l) g_k(z_l),
 * x_l in cell-local coordinates.  Sorted charges (t, q) and cell starts by
 * Morton key.  Writes level `depth` of Phi. */
void orc_p2m(int n, int depth, const double *st, const double *sq, const int64_t *start,
             double *Phi)
{
    const int64_t ncell = (int64_t)1 << (3 * depth);
    const int n3 = n * n * n, S = 1 << depth;
    double *P = Phi + level_offset(n, depth);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t key = 0; key < ncell; key++) {
        int cx, cy, cz;
        demorton3((uint32_t)key, depth, &cx, &cy, &cz);
        double *v = P + (((int64_t)cz * S + cy) * S + cx) * n3;
        for (int a = 0; a < n3; a++) v[a] = 0.0;
        for (int64_t s = start[key]; s < start[key + 1]; s++) {
            double gx[ORC_MAXN], gy[ORC_MAXN], gz[ORC_MAXN];
            orc_lagrange(n, st[3 * s], gx);
            orc_lagrange(n, st[3 * s + 1], gy);
            orc_lagrange(n, st[3 * s + 2], gz);
            for (int k = 0; k < n; k++)
                for (int j = 0; j < n; j++)
                    for (int i = 0; i < n; i++)
                        v[(k * n + j) * n + i] += sq[s] * gx[i] * gy[j] * gz[k];
        }
    }
}

/* One-dimensional shift along `axis` (eq. (threethree)): out = G (x) in on
 * every line of the n^3 vector parallel to the axis. */
static void shift_axis(int n, const double *G, int axis, const double *in, double *out)
{
    for (int k = 0; k < n; k++)
        for (int j = 0; j < n; j++)
            for (int i = 0; i < n; i++) {
                int idx[3] = {i, j, k};
                double s = 0.0;
                for (int m = 0; m < n; m++) {
                    int src[3] = {i, j, k};
                    src[axis] = m;
                    s += G[idx[axis] * n + m] * in[(src[2] * n + src[1]) * n + src[0]];
                }
                out[(k * n + j) * n + i] = s;
            }
}

/* §2.2 step 2: shift every cell's vector to its parent with the three
 * successive one-dimensional shifts of eq. (threethree) (x, then y, then z)
 * and sum the eight children; repeat from level `depth` up to level `lmin`. */
void orc_m2m(int n, int depth, int lmin, double *Phi)
{
    const int n3 = n * n * n;
    double G[2][ORC_MAXN * ORC_MAXN];
    orc_shift_matrix(n, 0, G[0]);
    orc_shift_matrix(n, 1, G[1]);
    for (int l = depth; l > lmin; l--) {
        const int S = 1 << l, Sp = S >> 1;
        const double *C = Phi + level_offset(n, l);
        double *P = Phi + level_offset(n, l - 1);
#pragma omp parallel for schedule(static)
        for (int64_t pc = 0; pc < (int64_t)Sp * Sp * Sp; pc++) {
            int px = (int)(pc % Sp), py = (int)((pc / Sp) % Sp), pz = (int)(pc / ((int64_t)Sp * Sp));
            double *v = P + pc * n3;
            double a[ORC_MAXN * ORC_MAXN * ORC_MAXN], b[ORC_MAXN * ORC_MAXN * ORC_MAXN];
            for (int e = 0; e < n3; e++) v[e] = 0.0;
            for (int hz = 0; hz < 2; hz++)
                for (int hy = 0; hy < 2; hy++)
                    for (int hx = 0; hx < 2; hx++) {
                        int cx = 2 * px + hx, cy = 2 * py + hy, cz = 2 * pz + hz;
                        const double *w = C + (((int64_t)cz * S + cy) * S + cx) * n3;
                        shift_axis(n, G[hx], 0, w, a);
                        shift_axis(n, G[hy], 1, a, b);
                        shift_axis(n, G[hz], 2, b, a);
                        for (int e = 0; e < n3; e++) v[e] += a[e];
                    }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* §2.2 step 3: downward pass                                                */
/* ------------------------------------------------------------------------ */

/* Transpose of the one-dimensional shift along `axis`: out = G^T (x) in. */
static void shift_axis_t(int n, const double *G, int axis, const double *in, double *out)
{
    for (int k = 0; k < n; k++)
        for (int j = 0; j < n; j++)
            for (int i = 0; i < n; i++) {
                int idx[3] = {i, j, k};
                double s = 0.0;
                for (int m = 0; m < n; m++) {
                    int src[3] = {i, j, k};
                    src[axis] = m;
                    s += G[m * n + idx[axis]] * in[(src[2] * n + src[1]) * n + src[0]];
                }
                out[(k * n + j) * n + i] = s;
            }
}

/* The interaction list of cell (cx, cy, cz) of a level with S cells per axis
 * (§2.2 step 3): the children of the parent cell and of its 26 neighbours
 * that are not adjacent to the cell (no offset with |o|_inf <= 1), in
 * (z, y, x) order of the source.  Open form: only sources inside the box;
 * periodic form: the source index wrapped, the offset kept.  Writes the
 * source cell (natural order (z S + y) S + x) and the offset's index
 * ((oz + 3) 7 + oy + 3) 7 + ox + 3 of every entry; returns their number. */
static int interaction_list(int S, int periodic, int cx, int cy, int cz, int64_t *src, int *oidx)
{
    const int px = cx >> 1, py = cy >> 1, pz = cz >> 1;
    int m = 0;
    for (int sz = 2 * (pz - 1); sz <= 2 * (pz + 1) + 1; sz++)
        for (int sy = 2 * (py - 1); sy <= 2 * (py + 1) + 1; sy++)
            for (int sx = 2 * (px - 1); sx <= 2 * (px + 1) + 1; sx++) {
                int ox = sx - cx, oy = sy - cy, oz = sz - cz;
                if (abs(ox) <= 1 && abs(oy) <= 1 && abs(oz) <= 1) continue;
                int wx = sx, wy = sy, wz = sz;
                if (periodic) {
                    wx = ((sx % S) + S) % S;
                    wy = ((sy % S) + S) % S;
                    wz = ((sz % S) + S) % S;
                } else if (sx < 0 || sy < 0 || sz < 0 || sx >= S || sy >= S || sz >= S) {
                    continue;
                }
                src[m] = ((int64_t)wz * S + wy) * S + wx;
                oidx[m] = ((oz + 3) * 7 + (oy + 3)) * 7 + (ox + 3);
                m++;
            }
    return m;
}

/* The list above for cell (cx, cy, cz) of level l (at most 189 entries). */
int orc_interaction_list(int l, int periodic, int cx, int cy, int cz, int64_t *src, int *oidx)
{
    return interaction_list(1 << l, periodic, cx, cy, cz, src, oidx);
}

/* The linear functional Psi_C(v) of §2.2 step 3 is stored as the vector L_C
 * with Psi_C(v) = L_C . v.
 *
 *  - Psi is zero at levels 0 and 1 (open form).  The periodic form (§4.2)
 *    starts at level 0 with the interaction of the box with its images beyond
 *    the 26 nearest (Ewald lattice kernel), and adds interaction lists from
 *    level 1 on, whose cells are the periodic images.
 *  - Psi_child(v) = Psi_parent(shift_{child->parent}(v)), i.e.
 *    L_child = shift^T L_parent.
 *  - B^n_{C,C~}(v, Phi_C~) is added for every C~ in the interaction list of C
 *    (eq. (bilinear)): L_C[a] += sum_b F(a, b~) Phi_C~[b], with
 *    F = 2^l / |a - b~| in unit-box units for cells of level l.
 *  - The interaction list (Greengard-Rokhlin, cited in §2.2): children of the
 *    parent's 26 neighbours and the parent itself that are not adjacent to C.
 *
 * need[l] (optional, natural index) marks the cells whose L is required;
 * the others are skipped.  Klat: the n^3 x n^3 lattice kernel (periodic). */
void orc_downward(int n, int depth, int periodic, const double *Phi, double *L,
                  const uint8_t *const *need, const double *Klat)
{
    const int n3 = n * n * n;
    double G[2][ORC_MAXN * ORC_MAXN];
    orc_shift_matrix(n, 0, G[0]);
    orc_shift_matrix(n, 1, G[1]);
    /* unit kernels K_o for the 7^3 offsets |o|_inf <= 3, stored transposed
     * (KT[b*n3 + a]) so that the accumulation below runs over b in order */
    double *KT = (double *)malloc(sizeof(double) * 343 * (size_t)n3 * n3);
    double *K = (double *)malloc(sizeof(double) * (size_t)n3 * n3);
    for (int oz = -3; oz <= 3; oz++)
        for (int oy = -3; oy <= 3; oy++)
            for (int ox = -3; ox <= 3; ox++) {
                int oi = ((oz + 3) * 7 + (oy + 3)) * 7 + (ox + 3);
                orc_m2l_kernel(n, ox, oy, oz, K);
                for (int a = 0; a < n3; a++)
                    for (int b = 0; b < n3; b++)
                        KT[(int64_t)oi * n3 * n3 + (int64_t)b * n3 + a] = K[(int64_t)a * n3 + b];
            }
    free(K);

    if (periodic) {
        /* level 0: the box against its far images */
        double *L0 = L + level_offset(n, 0);
        const double *P0 = Phi + level_offset(n, 0);
        for (int a = 0; a < n3; a++) {
            double s = 0.0;
            for (int b = 0; b < n3; b++) s += Klat[(int64_t)a * n3 + b] * P0[b];
            L0[a] = s;
        }
    } else {
        for (int e = 0; e < n3; e++) L[level_offset(n, 0) + e] = 0.0;
    }
    for (int l = 1; l <= depth; l++) {
        const int S = 1 << l, Sp = S >> 1;
        const double scale = level_scale(l);
        const double *Pl = Phi + level_offset(n, l);
        double *Ll = L + level_offset(n, l);
        const double *Lp = L + level_offset(n, l - 1);
        const int do_m2l = periodic ? (l >= 1) : (l >= 2);
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t c = 0; c < (int64_t)S * S * S; c++) {
            if (need && need[l] && !need[l][c]) continue;
            int cx = (int)(c % S), cy = (int)((c / S) % S), cz = (int)(c / ((int64_t)S * S));
            double *v = Ll + c * n3;
            /* Psi_child(v) = Psi_parent(shift(v)) */
            double a[ORC_MAXN * ORC_MAXN * ORC_MAXN], b[ORC_MAXN * ORC_MAXN * ORC_MAXN];
            int px = cx >> 1, py = cy >> 1, pz = cz >> 1;
            const double *w = Lp + (((int64_t)pz * Sp + py) * Sp + px) * n3;
            shift_axis_t(n, G[cz & 1], 2, w, a);
            shift_axis_t(n, G[cy & 1], 1, a, b);
            shift_axis_t(n, G[cx & 1], 0, b, a);
            for (int e = 0; e < n3; e++) v[e] = a[e];
            if (!do_m2l) continue;
            /* interaction list */
            int64_t il_src[189];
            int il_o[189];
            const int m = interaction_list(S, periodic, cx, cy, cz, il_src, il_o);
            for (int e = 0; e < m; e++) {
                const double *kt = KT + (int64_t)il_o[e] * n3 * n3;
                const double *src = Pl + il_src[e] * n3;
                for (int bb = 0; bb < n3; bb++) {
                    double f = scale * src[bb];
                    const double *row = kt + (int64_t)bb * n3;
                    for (int aa = 0; aa < n3; aa++) v[aa] += row[aa] * f;
                }
            }
        }
    }
    free(KT);
}

/* ------------------------------------------------------------------------ */
/* §2.2 steps 4-5 and the forces: far field at each charge, plus the near    */
/* field over the cell itself and its 26 neighbours                          */
/* ------------------------------------------------------------------------ */

/* Step 5 at sorted charge s: the direct sum over the charges of its cell and
 * of the 26 neighbours (no second neighbours, §1), skipping charges of the
 * same original particle (the split charges of one particle do not interact
 * with each other).  Coincident charges of different particles contribute
 * nothing and are counted in *coinc.  out = (phi per unit charge, F). */
static void near_field(int depth, int periodic, int64_t s, const double *st, const int32_t *scell,
                       const double *sq, const int64_t *sorigin, const int64_t *start,
                       double out[4], int64_t *coinc)
{
    const int S = 1 << depth;
    const double w = 1.0 / (double)S;
    int cx = scell[3 * s], cy = scell[3 * s + 1], cz = scell[3 * s + 2];
    double pn = 0.0, nfx = 0.0, nfy = 0.0, nfz = 0.0;
    for (int dz = -1; dz <= 1; dz++)
        for (int dy = -1; dy <= 1; dy++)
            for (int dx = -1; dx <= 1; dx++) {
                int nx = cx + dx, ny = cy + dy, nz = cz + dz;
                if (periodic) {
                    nx = (nx + S) % S;
                    ny = (ny + S) % S;
                    nz = (nz + S) % S;
                } else if (nx < 0 || ny < 0 || nz < 0 || nx >= S || ny >= S || nz >= S) {
                    continue;
                }
                uint32_t key = morton3(nx, ny, nz, depth);
                for (int64_t r = start[key]; r < start[key + 1]; r++) {
                    if (sorigin[r] == sorigin[s]) continue;
                    /* separation in unit-box units, neighbour cell at offset (dx,dy,dz) */
                    double rx = (st[3 * s] - st[3 * r] - dx) * w;
                    double ry = (st[3 * s + 1] - st[3 * r + 1] - dy) * w;
                    double rz = (st[3 * s + 2] - st[3 * r + 2] - dz) * w;
                    double r2 = rx * rx + ry * ry + rz * rz;
                    if (r2 == 0.0) {
                        (*coinc)++;
                        continue;
                    }
                    double rr = sqrt(r2);
                    /* pair potential q/r^g_power; force -q_s q_r grad_s (1/r^g_power) */
                    pn += g_power == 2 ? sq[r] / r2 : sq[r] / rr;
                    double c = g_power == 2 ? 2.0 * sq[s] * sq[r] / (r2 * r2)
                                            : sq[s] * sq[r] / (r2 * rr);
                    nfx += c * rx;
                    nfy += c * ry;
                    nfz += c * rz;
                }
            }
    out[0] = pn;
    out[1] = nfx;
    out[2] = nfy;
    out[3] = nfz;
}

/* For every sorted charge s (or those with mask[s] set):
 *   far:  phi_far = Psi_leaf(g(x_s)) = sum_ijk g_ijk(x_s) L_leaf[ijk]
 *         (step 4 per unit charge), and the force Psi_leaf(v'_a) with
 *         v'_a = -q d g / d a (end of §2.2);
 *   near: the direct sum over the charges of the same cell and of its 26
 *         neighbours (step 5; no second neighbours, §1), skipping charges of
 *         the same original particle (the split charges of one particle do
 *         not interact with each other).  Coincident charges of different
 *         particles contribute nothing and are counted in *ncoinc.
 * Outputs per charge (unit-box units): phi[s] per unit charge, F[3s..] force. */
void orc_evaluate(int n, int depth, int periodic, int64_t npts, const double *st,
                  const int32_t *scell, const double *sq, const int64_t *sorigin,
                  const int64_t *start, const double *L, const uint8_t *mask, double *phi,
                  double *F, int64_t *ncoinc)
{
    const int n3 = n * n * n, S = 1 << depth;
    const double *Ll = L + level_offset(n, depth);
    int64_t coinc = 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : coinc)
    for (int64_t s = 0; s < npts; s++) {
        if (mask && !mask[s]) continue;
        int cx = scell[3 * s], cy = scell[3 * s + 1], cz = scell[3 * s + 2];
        const double *v = Ll + (((int64_t)cz * S + cy) * S + cx) * n3;
        double gx[ORC_MAXN], gy[ORC_MAXN], gz[ORC_MAXN];
        double dx_[ORC_MAXN], dy_[ORC_MAXN], dz_[ORC_MAXN];
        orc_lagrange(n, st[3 * s], gx);
        orc_lagrange(n, st[3 * s + 1], gy);
        orc_lagrange(n, st[3 * s + 2], gz);
        orc_lagrange_deriv(n, st[3 * s], dx_);
        orc_lagrange_deriv(n, st[3 * s + 1], dy_);
        orc_lagrange_deriv(n, st[3 * s + 2], dz_);
        double pf = 0.0, gfx = 0.0, gfy = 0.0, gfz = 0.0;
        for (int k = 0; k < n; k++)
            for (int j = 0; j < n; j++)
                for (int i = 0; i < n; i++) {
                    double Lv = v[(k * n + j) * n + i];
                    pf += gx[i] * gy[j] * gz[k] * Lv;
                    gfx += dx_[i] * gy[j] * gz[k] * Lv;
                    gfy += gx[i] * dy_[j] * gz[k] * Lv;
                    gfz += gx[i] * gy[j] * dz_[k] * Lv;
                }
        /* d/du = 2^depth d/dt */
        double fx = -sq[s] * gfx * S, fy = -sq[s] * gfy * S, fz = -sq[s] * gfz * S;
        double nf[4];
        near_field(depth, periodic, s, st, scell, sq, sorigin, start, nf, &coinc);
        double pn = nf[0], nfx = nf[1], nfy = nf[2], nfz = nf[3];
        phi[s] = pf + pn;
        F[3 * s] = fx + nfx;
        F[3 * s + 1] = fy + nfy;
        F[3 * s + 2] = fz + nfz;
    }
    if (ncoinc) *ncoinc = coinc;
}

/* ------------------------------------------------------------------------ */
/* App. A.2: bilinear forms without shifts                                   */
/* ------------------------------------------------------------------------ */
/*
 * Every cell C's grid charges are taken with respect to the whole box S,
 * Phi^S_C = shift_{C->S}(Phi_C): the same vector as replacing C's point
 * charges directly with respect to S.  So the upward pass is a sum of the
 * children's vectors, and with
 *     BB_{C,C~}(v, w) = B_{C,C~}(shift_{S->C}(v), shift_{S->C~}(w))
 * the far field is a sum of BB over the interaction lists; the functional of
 * a cell, also taken with respect to S, passes to the children unchanged
 * (the downward pass is the identity).  shift_{S->C} is the inverse of
 * shift_{C->S}; it extrapolates from C to S and grows like 2^{l(n-1)}.
 */

/* shift_{C->S} along one axis for the cell of level l at coordinate c: C's
 * node a_i lies at (c + a_i)/2^l in box coordinates, and replacing a charge
 * there with respect to S gives the box weights g_b((c + a_i)/2^l).
 * G[b*n + i]. */
void orc_sf_shift_to_box(int n, int l, int c, double *G)
{
    double g[ORC_MAXN];
    const double h = ldexp(1.0, -l);
    for (int i = 0; i < n; i++) {
        orc_lagrange(n, h * ((double)c + tau(n, i)), g);
        for (int b = 0; b < n; b++) G[b * n + i] = g[b];
    }
}

/* Inverse of the n x n matrix A by Gauss-Jordan elimination with partial
 * pivoting; returns 0, or 1 if a pivot is zero. */
static int invert(int n, const double *A, double *X)
{
    double M[ORC_MAXN][2 * ORC_MAXN];
    for (int r = 0; r < n; r++)
        for (int c = 0; c < n; c++) {
            M[r][c] = A[r * n + c];
            M[r][n + c] = (r == c) ? 1.0 : 0.0;
        }
    for (int c = 0; c < n; c++) {
        int piv = c;
        for (int r = c + 1; r < n; r++)
            if (fabs(M[r][c]) > fabs(M[piv][c])) piv = r;
        if (M[piv][c] == 0.0) return 1;
        if (piv != c)
            for (int k = 0; k < 2 * n; k++) {
                double t = M[c][k];
                M[c][k] = M[piv][k];
                M[piv][k] = t;
            }
        double d = M[c][c];
        for (int k = 0; k < 2 * n; k++) M[c][k] /= d;
        for (int r = 0; r < n; r++) {
            if (r == c) continue;
            double f = M[r][c];
            if (f == 0.0) continue;
            for (int k = 0; k < 2 * n; k++) M[r][k] -= f * M[c][k];
        }
    }
    for (int r = 0; r < n; r++)
        for (int c = 0; c < n; c++) X[r * n + c] = M[r][n + c];
    return 0;
}

/* shift_{S->C} along one axis: the inverse of orc_sf_shift_to_box,
 * H[i*n + b] (cell node i, box node b).  Returns 0 or 1 (singular). */
int orc_sf_shift_from_box(int n, int l, int c, double *H)
{
    double G[ORC_MAXN * ORC_MAXN];
    orc_sf_shift_to_box(n, l, c, G);
    return invert(n, G, H);
}

/* Replacement of the charges of every finest cell directly with respect to
 * the box: Phi^S_leaf[i,j,k] = sum_l q_l g_i(X_l) g_j(Y_l) g_k(Z_l), X the
 * box coordinate (c + t)/2^depth of a charge at cell-local t.  Writes level
 * `depth` of PhiS (natural cell order). */
void orc_sf_p2m(int n, int depth, const double *st, const int32_t *scell, const double *sq,
                const int64_t *start, double *PhiS)
{
    const int64_t ncell = (int64_t)1 << (3 * depth);
    const int n3 = n * n * n, S = 1 << depth;
    const double h = 1.0 / (double)S;
    double *P = PhiS + level_offset(n, depth);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t key = 0; key < ncell; key++) {
        int cx, cy, cz;
        demorton3((uint32_t)key, depth, &cx, &cy, &cz);
        double *v = P + (((int64_t)cz * S + cy) * S + cx) * n3;
        for (int a = 0; a < n3; a++) v[a] = 0.0;
        for (int64_t s = start[key]; s < start[key + 1]; s++) {
            double gx[ORC_MAXN], gy[ORC_MAXN], gz[ORC_MAXN];
            orc_lagrange(n, h * ((double)scell[3 * s] + st[3 * s]), gx);
            orc_lagrange(n, h * ((double)scell[3 * s + 1] + st[3 * s + 1]), gy);
            orc_lagrange(n, h * ((double)scell[3 * s + 2] + st[3 * s + 2]), gz);
            for (int k = 0; k < n; k++)
                for (int j = 0; j < n; j++)
                    for (int i = 0; i < n; i++)
                        v[(k * n + j) * n + i] += sq[s] * gx[i] * gy[j] * gz[k];
        }
    }
}

/* Upward pass of App. A.2: Phi^S_parent = sum of the eight children's Phi^S,
 * from level `depth` up to level `lmin`. */
void orc_sf_upward(int n, int depth, int lmin, double *PhiS)
{
    const int n3 = n * n * n;
    for (int l = depth; l > lmin; l--) {
        const int S = 1 << l, Sp = S >> 1;
        const double *C = PhiS + level_offset(n, l);
        double *P = PhiS + level_offset(n, l - 1);
#pragma omp parallel for schedule(static)
        for (int64_t pc = 0; pc < (int64_t)Sp * Sp * Sp; pc++) {
            int px = (int)(pc % Sp), py = (int)((pc / Sp) % Sp), pz = (int)(pc / ((int64_t)Sp * Sp));
            double *v = P + pc * n3;
            for (int e = 0; e < n3; e++) v[e] = 0.0;
            for (int hz = 0; hz < 2; hz++)
                for (int hy = 0; hy < 2; hy++)
                    for (int hx = 0; hx < 2; hx++) {
                        int cx = 2 * px + hx, cy = 2 * py + hy, cz = 2 * pz + hz;
                        const double *w = C + (((int64_t)cz * S + cy) * S + cx) * n3;
                        for (int e = 0; e < n3; e++) v[e] += w[e];
                    }
        }
    }
}

/* out = BB v for the cells C~ (target, coordinates ct) and C (source, cs) of
 * level l at offset o = C - C~ before any periodic wrap: the box-basis
 * vector v of C is shifted to C (shift_{S->C}), the bilinear form of the two
 * unit cells at offset o, scaled by 2^l to unit-box units, is applied, and
 * the result is taken back to the box basis with the transpose of
 * shift_{S->C~}.  Hs/Ht: the per-axis shift_{S->C} matrices of source and
 * target (orc_sf_shift_from_box); K: the unit kernel of offset o. */
static void sf_apply(int n, int l, const double *const Hs[3], const double *const Ht[3],
                     const double *K, const double *v, double *out)
{
    const int n3 = n * n * n;
    double a[ORC_MAXN * ORC_MAXN * ORC_MAXN], b[ORC_MAXN * ORC_MAXN * ORC_MAXN];
    shift_axis(n, Hs[0], 0, v, a);
    shift_axis(n, Hs[1], 1, a, b);
    shift_axis(n, Hs[2], 2, b, a);
    const double scale = ldexp(1.0, l);
    for (int r = 0; r < n3; r++) {
        double s = 0.0;
        for (int c = 0; c < n3; c++) s += K[(int64_t)r * n3 + c] * a[c];
        b[r] = scale * s;
    }
    shift_axis_t(n, Ht[0], 0, b, a);
    shift_axis_t(n, Ht[1], 1, a, b);
    shift_axis_t(n, Ht[2], 2, b, out);
}

/* The matrix of BB for target cell ct, source cell cs (wrapped coordinates)
 * at offset o, level l: B[r*n^3 + c] = (BB e_c)[r], box-node indices.
 * Returns 0, or 1 if a shift is singular. */
int orc_sf_bilinear(int n, int l, const int *ct, const int *cs, const int *o, double *B)
{
    const int n3 = n * n * n;
    double hs[3][ORC_MAXN * ORC_MAXN], ht[3][ORC_MAXN * ORC_MAXN];
    for (int ax = 0; ax < 3; ax++)
        if (orc_sf_shift_from_box(n, l, cs[ax], hs[ax]) || orc_sf_shift_from_box(n, l, ct[ax], ht[ax]))
            return 1;
    const double *Hs[3] = {hs[0], hs[1], hs[2]}, *Ht[3] = {ht[0], ht[1], ht[2]};
    double *K = (double *)malloc(sizeof(double) * (size_t)n3 * n3);
    double *e = (double *)calloc((size_t)n3, sizeof(double));
    double *col = (double *)malloc(sizeof(double) * (size_t)n3);
    orc_m2l_kernel(n, o[0], o[1], o[2], K);
    for (int c = 0; c < n3; c++) {
        e[c] = 1.0;
        sf_apply(n, l, Hs, Ht, K, e, col);
        e[c] = 0.0;
        for (int r = 0; r < n3; r++) B[(int64_t)r * n3 + c] = col[r];
    }
    free(K);
    free(e);
    free(col);
    return 0;
}

/* Downward pass of App. A.2 on box-basis functionals L^S:
 *   level 0: zero (open form), or the box against its far images (periodic
 *            form, §4.2: the box basis is the level-0 cell's basis);
 *   level l: L^S_C~ = L^S_parent (the identity) + sum over the interaction
 *            list of BB_{C~,C} Phi^S_C, the same lists as orc_downward.
 * need[l] as in orc_downward.  Returns 0, or 1 if a shift is singular. */
int orc_sf_downward(int n, int depth, int periodic, const double *PhiS, double *LS,
                    const uint8_t *const *need, const double *Klat)
{
    const int n3 = n * n * n;
    if (periodic) {
        double *L0 = LS + level_offset(n, 0);
        const double *P0 = PhiS + level_offset(n, 0);
        for (int a = 0; a < n3; a++) {
            double s = 0.0;
            for (int b = 0; b < n3; b++) s += Klat[(int64_t)a * n3 + b] * P0[b];
            L0[a] = s;
        }
    } else {
        for (int e = 0; e < n3; e++) LS[level_offset(n, 0) + e] = 0.0;
    }
    /* unit kernels K_o, |o|_inf <= 3 */
    double *Kall = (double *)malloc(sizeof(double) * 343 * (size_t)n3 * n3);
    for (int oi = 0; oi < 343; oi++)
        orc_m2l_kernel(n, oi % 7 - 3, (oi / 7) % 7 - 3, oi / 49 - 3, Kall + (int64_t)oi * n3 * n3);
    int bad = 0;
    for (int l = 1; l <= depth; l++) {
        const int S = 1 << l, Sp = S >> 1;
        const double *Pl = PhiS + level_offset(n, l);
        double *Ll = LS + level_offset(n, l);
        const double *Lp = LS + level_offset(n, l - 1);
        const int do_m2l = periodic ? (l >= 1) : (l >= 2);
        /* shift_{S->C} per axis coordinate of this level */
        double *H = (double *)malloc(sizeof(double) * (size_t)S * n * n);
        for (int c = 0; c < S; c++) bad |= orc_sf_shift_from_box(n, l, c, H + (size_t)c * n * n);
#pragma omp parallel for schedule(dynamic, 16)
        for (int64_t c = 0; c < (int64_t)S * S * S; c++) {
            if (need && need[l] && !need[l][c]) continue;
            int cx = (int)(c % S), cy = (int)((c / S) % S), cz = (int)(c / ((int64_t)S * S));
            double *v = Ll + c * n3;
            int px = cx >> 1, py = cy >> 1, pz = cz >> 1;
            const double *w = Lp + (((int64_t)pz * Sp + py) * Sp + px) * n3;
            for (int e = 0; e < n3; e++) v[e] = w[e];
            if (!do_m2l) continue;
            const double *Ht[3] = {H + (size_t)cx * n * n, H + (size_t)cy * n * n,
                                   H + (size_t)cz * n * n};
            double y[ORC_MAXN * ORC_MAXN * ORC_MAXN];
            int64_t il_src[189];
            int il_o[189];
            const int m = interaction_list(S, periodic, cx, cy, cz, il_src, il_o);
            for (int k = 0; k < m; k++) {
                        const int wx = (int)(il_src[k] % S), wy = (int)((il_src[k] / S) % S),
                                  wz = (int)(il_src[k] / ((int64_t)S * S));
                        const double *Hs[3] = {H + (size_t)wx * n * n, H + (size_t)wy * n * n,
                                               H + (size_t)wz * n * n};
                        const double *src = Pl + il_src[k] * n3;
                        sf_apply(n, l, Hs, Ht, Kall + (int64_t)il_o[k] * n3 * n3, src, y);
                        for (int e = 0; e < n3; e++) v[e] += y[e];
                    }
        }
        free(H);
    }
    free(Kall);
    return bad;
}

/* Steps 4-5 with box-basis functionals: the far field at a charge is
 * L^S_leaf . g(X) with the box weights at its box coordinate X = (c + t)/2^depth,
 * and the far force -q dg/dX (box coordinates are unit-box units); the near
 * field as orc_evaluate. */
void orc_sf_evaluate(int n, int depth, int periodic, int64_t npts, const double *st,
                     const int32_t *scell, const double *sq, const int64_t *sorigin,
                     const int64_t *start, const double *LS, const uint8_t *mask, double *phi,
                     double *F, int64_t *ncoinc)
{
    const int n3 = n * n * n, S = 1 << depth;
    const double h = 1.0 / (double)S;
    const double *Ll = LS + level_offset(n, depth);
    int64_t coinc = 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : coinc)
    for (int64_t s = 0; s < npts; s++) {
        if (mask && !mask[s]) continue;
        int cx = scell[3 * s], cy = scell[3 * s + 1], cz = scell[3 * s + 2];
        const double *v = Ll + (((int64_t)cz * S + cy) * S + cx) * n3;
        double X = h * ((double)cx + st[3 * s]), Y = h * ((double)cy + st[3 * s + 1]),
               Z = h * ((double)cz + st[3 * s + 2]);
        double gx[ORC_MAXN], gy[ORC_MAXN], gz[ORC_MAXN];
        double dx_[ORC_MAXN], dy_[ORC_MAXN], dz_[ORC_MAXN];
        orc_lagrange(n, X, gx);
        orc_lagrange(n, Y, gy);
        orc_lagrange(n, Z, gz);
        orc_lagrange_deriv(n, X, dx_);
        orc_lagrange_deriv(n, Y, dy_);
        orc_lagrange_deriv(n, Z, dz_);
        double pf = 0.0, gfx = 0.0, gfy = 0.0, gfz = 0.0;
        for (int k = 0; k < n; k++)
            for (int j = 0; j < n; j++)
                for (int i = 0; i < n; i++) {
                    double Lv = v[(k * n + j) * n + i];
                    pf += gx[i] * gy[j] * gz[k] * Lv;
                    gfx += dx_[i] * gy[j] * gz[k] * Lv;
                    gfy += gx[i] * dy_[j] * gz[k] * Lv;
                    gfz += gx[i] * gy[j] * dz_[k] * Lv;
                }
        double nf[4];
        near_field(depth, periodic, s, st, scell, sq, sorigin, start, nf, &coinc);
        phi[s] = pf + nf[0];
        F[3 * s] = -sq[s] * gfx + nf[1];
        F[3 * s + 1] = -sq[s] * gfy + nf[2];
        F[3 * s + 2] = -sq[s] * gfz + nf[3];
    }
    if (ncoinc) *ncoinc = coinc;
}

/* Steps 4-5 with the forces taken from the force kernels (§4.1's remark):
 * L holds the potential functionals, LF[c] those of the c-th force component
 * (orc_set_kernel(c + 1) for the downward pass).  Far potential per unit
 * charge g(x).L_leaf as in orc_evaluate; far force component c is
 * q g(x).LF[c]_leaf with the plain weights; the near field as orc_evaluate. */
void orc_evaluate_kernel(int n, int depth, int periodic, int64_t npts, const double *st,
                         const int32_t *scell, const double *sq, const int64_t *sorigin,
                         const int64_t *start, const double *L, const double *LFx,
                         const double *LFy, const double *LFz, const uint8_t *mask, double *phi,
                         double *F, int64_t *ncoinc)
{
    const int n3 = n * n * n, S = 1 << depth;
    const int64_t off = level_offset(n, depth);
    const double *LF[3] = {LFx + off, LFy + off, LFz + off};
    int64_t coinc = 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : coinc)
    for (int64_t s = 0; s < npts; s++) {
        if (mask && !mask[s]) continue;
        int cx = scell[3 * s], cy = scell[3 * s + 1], cz = scell[3 * s + 2];
        const int64_t cell = (((int64_t)cz * S + cy) * S + cx) * n3;
        double gx[ORC_MAXN], gy[ORC_MAXN], gz[ORC_MAXN];
        orc_lagrange(n, st[3 * s], gx);
        orc_lagrange(n, st[3 * s + 1], gy);
        orc_lagrange(n, st[3 * s + 2], gz);
        double pf = 0.0, f[3] = {0.0, 0.0, 0.0};
        for (int k = 0; k < n; k++)
            for (int j = 0; j < n; j++)
                for (int i = 0; i < n; i++) {
                    int a = (k * n + j) * n + i;
                    double w = gx[i] * gy[j] * gz[k];
                    pf += w * L[off + cell + a];
                    for (int c = 0; c < 3; c++) f[c] += w * LF[c][cell + a];
                }
        double nf[4];
        near_field(depth, periodic, s, st, scell, sq, sorigin, start, nf, &coinc);
        phi[s] = pf + nf[0];
        for (int c = 0; c < 3; c++) F[3 * s + c] = sq[s] * f[c] + nf[1 + c];
    }
    if (ncoinc) *ncoinc = coinc;
}

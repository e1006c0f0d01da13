/*
 * fmm_gb300.h — C ABI of the GB300 (sm_103a) replacement-based fast multipole
 * method of Y. Kajima, "Notes on the Fast Multipole Method" (arXiv:2212.13080).
 *
 * The method (§2.2) computes, for N point charges in a cubic box, the Coulomb
 * potential of every charge, the total energy and the forces:
 *   - the box is divided into an octree of depth `depth` (§2.2 step 1);
 *   - the charges of every finest cell are replaced by p^3 charges on the
 *     cell's p-division points (replacement, eq. ex66), shifted up the tree
 *     (shift, eq. threethree);
 *   - well-separated cells interact through the p^3 x p^3 bilinear form of the
 *     grid charges (eq. bilinear), passed down the tree as linear functionals
 *     (§2.2 step 3) and evaluated at the charges (step 4, and the far-field
 *     force at the end of §2.2);
 *   - the near field is summed directly over each finest cell's 27-cell
 *     neighbourhood (step 5).
 * The continuous form (§2.3) first splits every charge that lies closer than
 * d to a plane of the finest cells into p (p^2, p^3) charges on a segment of
 * length 2d across the plane; the periodic form (§4.2) also splits at the box
 * walls and adds the lattice sum of the box's far images (Ewald, tin-foil).
 *
 * Conventions shared by every entry point:
 *   - Every function returns an int status: FMM_OK (0) or one FMM_ERR_* code.
 *     No C++ exception crosses this boundary.  fmm_strerror() names a code.
 *   - Device pointers are CUDA device (or managed) memory of the current
 *     device; the caller owns them.  Host pointers are marked "host".
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default).
 *     All device work of a call is queued on it, in order.
 *   - Positions are float32, row-major (n, 3): x0 y0 z0 x1 y1 z1 ...
 *     Charges are float32 (n).  Output arrays are float32, or float64 when
 *     the plan's precision is FMM_PREC_FP64.
 *   - Units: potential phi_i = sum_{j != i} q_j / r_ij (per unit charge),
 *     energy E = 1/2 sum_i q_i phi_i, force F_i = -dE/dx_i, in the units of
 *     the positions and charges (Coulomb constant 1, §3.1).
 */
#ifndef FMM_GB300_H
#define FMM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define FMM_OK 0
#define FMM_ERR_ARG 1            /* invalid argument (depth, p, box, sizes, null) */
#define FMM_ERR_OOM 2            /* device allocation failed, or plan too large */
#define FMM_ERR_OUT_OF_BOX 3     /* open form: a position outside [x0, x0+L) */
#define FMM_ERR_NONFINITE 4      /* a position is NaN or infinite */
#define FMM_ERR_SPLIT_OVERFLOW 5 /* continuous form: more split charges than the
                                    workspace was sized for (fmm_opts_t.split_capacity) */
#define FMM_ERR_TIMEOUT 6        /* a bounded device-side wait gave up */
#define FMM_ERR_CUDA 7           /* a CUDA runtime call failed */
#define FMM_ERR_STATE 8          /* fmm_backward without a matching fmm_eval */
#define FMM_ERR_WORKSPACE 9      /* workspace pointer null, misaligned or too small */
#define FMM_ERR_UNSUPPORTED 10   /* combination not built (e.g. tensor-core M2L for this p) */

/* ---- precision of the far-field contraction (and of everything else) ----- */
#define FMM_PREC_FP32 0   /* FP32 everywhere (SIMT bilinear forms) */
#define FMM_PREC_FP64 1   /* FP64 everywhere; outputs are float64 */
#define FMM_PREC_TF32X3 2 /* bilinear forms on tcgen05 tensor cores, 3-pass split TF32,
                             FP32 accumulate; rest FP32 */
#define FMM_PREC_TF32X1 3 /* tensor cores, one TF32 pass (10-bit mantissa operands),
                             FP32 accumulate; rest FP32 */
#define FMM_PREC_BF16X3 4 /* tensor cores, 3-pass split BF16 (hi = bf16(x),
                             lo = bf16(x - hi)), FP32 accumulate; rest FP32 */

/* ---- flags of fmm_eval ---------------------------------------------------- */
#define FMM_FORCE_ADJOINT 0 /* forces = -dE/dx of the FMM energy (default) */
#define FMM_FORCE_PAPER 1   /* split axes: sum of the forces the split charges feel (§2.3) */
#define FMM_KERNEL_COULOMB 0
#define FMM_KERNEL_INV_SQUARE 1
#define FMM_FORCE_KERNEL 2  /* far forces from the force kernels r/|r|^3 (§4.1, other
                               kernels): three more functionals per cell through the same
                               interaction lists (periodic: the gradient of the lattice term),
                               read with the plain weights; a particle's force is the sum of
                               its charges' forces.  Conserves total momentum exactly; the
                               backward pass stays the adjoint -dE/dx.  Not with shift_free. */

typedef struct fmm_plan_s *fmm_plan_t;

typedef struct {
    int continuous;        /* 1: split near the planes of the finest cells (§2.3, §4.2) */
    double split_ratio;    /* d / finest-cell width, in (0, 0.5); <= 0 selects 1/256
                              (2d = w/128; §3.2 uses 2d = 1/1024 with w = 1/8) */
    double split_capacity; /* workspace holds split_capacity * n charges after the split;
                              <= 0 selects max(2, 1.5 (1 + 2 (d/w)(m-1))^3), m = p
                              (even p) or p+1 (odd p): 1.5x the uniform-density mean */
    int precision;         /* FMM_PREC_* */
    int force_mode;        /* FMM_FORCE_ADJOINT, FMM_FORCE_PAPER or FMM_FORCE_KERNEL */
    int sync;              /* 1 (default when opts is NULL): fmm_eval waits for the device
                              and returns device-side errors; 0: fmm_eval returns after
                              queueing, fmm_status() reports them later */
    double grid_scale;     /* spacing of the p-division points in units of the standard
                              arrangement i/(p-1), about the cell centre (§4.1: the
                              "reduced" arrangement, e.g. 1/1.2); (0, 1]; <= 0 selects 1;
                              plain form only (continuous with a scale != 1:
                              FMM_ERR_UNSUPPORTED) */
    int shift_free;        /* 1: App. A.2, bilinear forms without shifts.  Every cell's grid
                              charges and functional are taken with respect to the box (the
                              upward pass sums children, the downward pass is the identity),
                              and the plan precomputes, on the device in FP64, one matrix
                              BB = shift_{S->C~}^T K_o shift_{S->C} per (cell, interaction-list
                              offset) of every level: 8 p^6 bytes each, plan-owned.
                              shift_{S->C} extrapolates over 2^l cells, so the forms lose
                              about 2(p-1) bits per level: FMM_PREC_FP64 only, p <= 5, and
                              tables of at most 32 GiB (else FMM_ERR_UNSUPPORTED); the
                              reduced arrangement and batched plans are not supported.
                              0 (default): the shifted form of §2.2. */
    int kernel;            /* FMM_KERNEL_COULOMB (default): F(P, P~) = 1/|P - P~|;
                              FMM_KERNEL_INV_SQUARE: 1/|P - P~|^2, the other function §4.1
                              names, for the far forms and the near field alike (potential
                              sum_j q_j/r^2, force 2 q_i q_j r/r^4).  Open boundary only (its
                              lattice sum diverges) and not with shift_free
                              (FMM_ERR_UNSUPPORTED). */
} fmm_opts_t;

/* Fills *opts with the defaults (continuous 0, split_ratio 1/256, split_capacity 0
 * (automatic), precision FP32, adjoint forces, sync 1, grid_scale 1, shift_free 0,
 * kernel FMM_KERNEL_COULOMB). */
void fmm_opts_default(fmm_opts_t *opts);

/*
 * fmm_plan_create — build the tables of one (box, depth, p, form) (§2.1, §2.2).
 *   box     host, 4 doubles: x0, y0, z0 (lower corner) and edge length L > 0.
 *   depth   octree depth l_f, 2 <= depth <= 8 (§2.2 step 1 needs l_f >= 2).
 *   p       points per cell edge (the paper's order n), 2 <= p <= 8.
 *   periodic 0: open boundary; 1: periodic box (§4.2).
 *   opts    host, nullable (defaults).
 *   max_n   largest particle count fmm_eval will be given with this plan.
 * Builds in FP64 on the host: the p-division points and Lagrange coefficients,
 * the two child->parent shift matrices (eq. trans), the 316 unit-cell
 * bilinear-form kernels 1/|a - (o + b)| for |o|_inf <= 3 (eq. bilinear), and
 * (periodic) the Ewald lattice kernel of the box's far images; uploads them to
 * the current device.  The plan owns those tables (device memory freed by
 * fmm_plan_destroy).  With opts.shift_free it also builds the per-axis
 * shift_{S->C} matrices and computes the App. A.2 forms on the device (FP64,
 * synchronous).  Errors: FMM_ERR_ARG, FMM_ERR_OOM, FMM_ERR_CUDA,
 * FMM_ERR_UNSUPPORTED.
 */
int fmm_plan_create(fmm_plan_t *plan, const double box[4], int depth, int p, int periodic,
                    const fmm_opts_t *opts, int64_t max_n);

/* Frees the plan's device tables.  NULL is accepted. */
void fmm_plan_destroy(fmm_plan_t plan);

/*
 * fmm_workspace_size — bytes of device workspace fmm_eval needs for n
 * particles (n <= max_n).  The workspace holds the sorted charges, the grid
 * charges Phi and functionals L of every level, and the status word; it is
 * the caller's memory (any 256-byte aligned device allocation) and it is the
 * state fmm_backward reuses.  Errors: FMM_ERR_ARG.
 */
int fmm_workspace_size(fmm_plan_t plan, int64_t n, size_t *bytes);

/*
 * fmm_eval — one evaluation of §2.2 (+ §2.3 split, §4.2 periodic).
 *   n          number of particles, 0 <= n <= max_n (n = 0: energy 0).
 *   pos        device, float32 (n,3).  Open form: every position must lie in
 *              [x0, x0+L)^3 (else FMM_ERR_OUT_OF_BOX); periodic: wrapped.
 *   q          device, float32 (n).
 *   potential  device, (n) float32 (float64 for FP64 plans), nullable.
 *   energy     device, 1 double, nullable.
 *   forces     device, (n,3) float32 (float64 for FP64 plans), nullable.
 *   workspace  device, >= fmm_workspace_size(plan, n) bytes, 256-byte aligned.
 *   stream     cudaStream_t as void*.
 * With opts.sync = 1 the call waits for the device and returns the device
 * status (FMM_ERR_OUT_OF_BOX, FMM_ERR_NONFINITE, FMM_ERR_SPLIT_OVERFLOW);
 * outputs are then undefined if the status is not FMM_OK.  A stream being
 * captured into a CUDA graph cannot be waited on: with opts.sync = 1 the call
 * then returns FMM_ERR_ARG before any work (plans for captured streams take
 * opts.sync = 0 and read the status later with fmm_status).
 */
int fmm_eval(fmm_plan_t plan, int64_t n, const float *pos, const float *q, void *potential,
             double *energy, void *forces, void *workspace, size_t workspace_bytes,
             void *stream);

/*
 * fmm_backward — adjoint of the energy (end of §2.2; forces as -dE/dx):
 * grad_pos = -F * grad_energy, grad_q = phi * grad_energy, recomputing only the
 * per-charge far-field gradients and near-field forces from the tree, grid
 * charges and functionals that the last fmm_eval on this workspace left in it
 * (no binning, sort, upward or downward pass).
 *   grad_energy  device, 1 double (dLoss/dE).
 *   grad_pos     device, (n,3) float32 (float64 for FP64 plans), nullable.
 *   grad_q       device, (n) float32 (float64 for FP64 plans), nullable.
 * pos and q must be the arrays the last fmm_eval was given.  Errors:
 * FMM_ERR_STATE if the workspace holds no evaluation of this plan and n: the
 * host checks that this plan's last fmm_eval used this workspace and n, and
 * the device checks the tag (plan, n) that every evaluation leaves in the
 * workspace header, so an evaluation of another plan into the same workspace
 * since then is caught too (returned with opts.sync = 1, else by fmm_status;
 * the gradients are then undefined).
 */
int fmm_backward(fmm_plan_t plan, int64_t n, const float *pos, const float *q,
                 const double *grad_energy, void *grad_pos, void *grad_q, void *workspace,
                 size_t workspace_bytes, void *stream);

/*
 * fmm_status — device-side status of the last fmm_eval/fmm_backward on this
 * workspace (waits on `stream`).  For opts.sync = 0.  workspace NULL: the
 * scratch array of fmm_eval_static on the current device.
 */
int fmm_status(fmm_plan_t plan, const void *workspace, void *stream);

/*
 * fmm_debug_dump — copies one intermediate of the last evaluation on
 * `workspace` to host memory `dst` (host, `bytes` long), after waiting on
 * `stream`.  Layouts:
 *   FMM_DUMP_COUNTS   int32 [4]: n, number of charges after the split, number of
 *                     finest cells, number of coincident pairs skipped
 *   FMM_DUMP_KEYS     uint32 [n_eff]: Morton key of each charge, emitted order
 *   FMM_DUMP_ORIGIN   int32 [n_eff]: particle of each charge, sorted order
 *   FMM_DUMP_PERM     int32 [n_eff]: emitted index of each sorted slot
 *   FMM_DUMP_START    int32 [cells+1]: first sorted slot of each finest cell (Morton)
 *   FMM_DUMP_POINTS   real [n_eff][4]: (t_x, t_y, t_z, q_eff) per sorted slot,
 *                     t in finest-cell units (real = float, double for FP64 plans)
 *   FMM_DUMP_PHI      real [level][8^level][p^3]: grid charges, natural cell
 *                     order (cz*S + cy)*S + cx, levels 0..depth (shift-free plans:
 *                     the box-basis charges Phi^S of App. A.2); the open form
 *                     forms them from level 2, levels 0 and 1 read as zero
 *   FMM_DUMP_LOCAL    real, same layout: functionals L (Psi_C(v) = L_C . v) of
 *                     the potential kernel (force-kernel plans keep three more
 *                     blocks, not dumped; shift-free plans: box-basis L^S).
 *                     They are formed only at cells that hold charges (step 4
 *                     reads no other) on the levels of the downward pass (open
 *                     form: levels >= 2); every other entry reads as zero.
 *   FMM_DUMP_OUT      real [n_eff][4]: (phi, F_x, F_y, F_z) per sorted charge in
 *                     unit-box units (phi per unit charge, F with the charge)
 * Errors: FMM_ERR_ARG (unknown item or dst too small).
 */
#define FMM_DUMP_COUNTS 0
#define FMM_DUMP_KEYS 1
#define FMM_DUMP_ORIGIN 2
#define FMM_DUMP_PERM 3
#define FMM_DUMP_START 4
#define FMM_DUMP_POINTS 5
#define FMM_DUMP_PHI 6
#define FMM_DUMP_LOCAL 7
#define FMM_DUMP_OUT 8
#define FMM_DUMP_WAIT 9
int fmm_debug_dump(fmm_plan_t plan, int what, const void *workspace, void *dst, size_t bytes,
                   void *stream);

/* Bytes fmm_debug_dump needs for `what` after the last evaluation on
 * `workspace` (waits on `stream`). */
int fmm_debug_size(fmm_plan_t plan, int what, const void *workspace, size_t *bytes,
                   void *stream);

/*
 * Failure-detection test hook (the paper has no counterpart).  With
 * FMM_INJECT_TC_STALL the next fmm_eval of the plan runs its tensor-core
 * contraction with the producer arming the first stage's barrier without
 * issuing that stage's copies: the barrier's transaction count is never met,
 * the consumer's bounded wait (about 2 s of SM clock) expires, the kernel
 * records the wait site in the workspace header, waits for its own copies and
 * MMAs, frees its tensor memory and returns, and the call returns
 * FMM_ERR_TIMEOUT.  No fault, trap or unbounded wait: the context stays usable.
 * The hook disarms itself after one evaluation; FMM_INJECT_NONE disarms it.
 * Plans without tensor-core contraction (FP32, FP64) return FMM_ERR_UNSUPPORTED.
 * The wait site: fmm_debug_dump(FMM_DUMP_WAIT) = int[4] (site: 1 producer slot,
 * 2 MMA region, 3 MMA operands, 4 epilogue region, 0 none; block; level;
 * iteration).
 */
#define FMM_INJECT_NONE 0
#define FMM_INJECT_TC_STALL 1
int fmm_debug_inject(fmm_plan_t plan, int what);

/*
 * Stage timing and launch accounting (tracing).
 * fmm_set_timing(plan, 1) makes every later fmm_eval/fmm_backward of the plan
 * bracket each stage's kernels with CUDA events on the call's stream;
 * fmm_get_stats() waits for them and reports the device time per stage (ms)
 * of the last call, and the number of kernels that call launched (counted
 * whether or not timing is on).  Stage ids: FMM_STAGE_*.
 * on = 2 also runs every stage on the call's stream (the near field and the
 * coarse levels are otherwise overlapped with the far field on plan-owned
 * streams), so that each stage's time is its kernels' own duration; results
 * are identical.  on = 0 switches timing off.
 */
#define FMM_STAGE_BIN 0      /* binning and split (§2.2 step 1, §2.3) */
#define FMM_STAGE_SORT 1     /* finest-cell ranges and stable sort */
#define FMM_STAGE_P2M 2      /* replacement at the finest cells (eq. ex66) */
#define FMM_STAGE_M2M 3      /* shifts upward (eq. threethree) and halo */
#define FMM_STAGE_M2L 4      /* bilinear forms of the interaction lists, lattice term */
#define FMM_STAGE_L2L 5      /* shift transposes downward */
#define FMM_STAGE_L2P 6      /* far field at the charges */
#define FMM_STAGE_P2P 7      /* near field over 27 cells */
#define FMM_STAGE_UNSPLIT 8  /* recombination, outputs, FP64 energy */
#define FMM_NSTAGES 9
typedef struct {
    int launches;                    /* kernels launched by the last call */
    int timed;                       /* 1 if stage_ms is valid */
    double stage_ms[FMM_NSTAGES];    /* device time per stage of the last call */
} fmm_stats_t;
int fmm_set_timing(fmm_plan_t plan, int on);
int fmm_get_stats(fmm_plan_t plan, fmm_stats_t *stats);

/*
 * Batched evaluation of many independent systems (each its own box, depth
 * and particle count; one p, form and precision for all), for ensembles of
 * small systems whose separate evaluations would be launch-bound.  Each
 * system is §2.2 (+ §2.3, §4.2) exactly as fmm_eval computes it.
 *
 * fmm_batch_create — nsys systems: boxes (host, nsys x 4: x0, y0, z0, L),
 *   depths (host, nsys), max_n (host, nsys); p, periodic and opts as
 *   fmm_plan_create (opts.sync is honoured; opts applies to every system).
 *   Systems of the same depth share one set of tables.  Errors as
 *   fmm_plan_create.
 */
typedef struct fmm_batch_s *fmm_batch_t;
int fmm_batch_create(fmm_batch_t *batch, int nsys, const double *boxes, const int *depths, int p,
                     int periodic, const fmm_opts_t *opts, const int64_t *max_n);
void fmm_batch_destroy(fmm_batch_t batch);

/* Bytes of device workspace for particle counts n (host, nsys). */
int fmm_batch_workspace_size(fmm_batch_t batch, const int64_t *n, size_t *bytes);

/*
 * fmm_batch_eval — evaluates every system.  Particles of system i are rows
 * offsets[i] .. offsets[i+1]-1 (offsets: host, nsys + 1, CSR) of pos (device,
 * float32 (N,3)), q, potential and forces (as fmm_eval); energy: device,
 * nsys doubles (nullable).  Every kernel launch site of an evaluation runs
 * once for all systems: each system's launch parameters are recorded, and
 * one launch of the site covers every system's blocks (a block finds its
 * system from the prefix of the systems' block counts), so each system's
 * results equal its single-system evaluation bit for bit.  The merged
 * launches are captured once into a CUDA graph and replayed by later calls
 * with the same pointers and counts (one graph launch per call); the first
 * call times the schedules (one stream, or the near field on a second stream)
 * and keeps the faster (fmm_batch_get_stats reports it).  Batches whose
 * systems' launch sequences do not merge (FP64 plans) run as per-system
 * pipelines spread over stream lanes instead, their count chosen the same
 * way.  Returns the first device-side error of any system (opts.sync = 1).
 */
int fmm_batch_eval(fmm_batch_t batch, const int64_t *offsets, const float *pos, const float *q,
                   void *potential, double *energy, void *forces, void *workspace,
                   size_t workspace_bytes, void *stream);

/* launches: kernels launched by the last fmm_batch_eval (inside its graph);
 * merged: 1 if every call site ran as one launch for all systems; schedule:
 * the merged form's schedule chosen by the autotuner (0: one stream, 1: the
 * near field on a second stream beside the rest); lanes: stream lanes of the
 * per-system form (0 when merged); graph: 1 if the last call replayed a
 * captured graph. */
typedef struct {
    int launches;
    int lanes;
    int graph;
    double tune_ms[8];  /* ms per call measured on the first call: lanes = 2, 4, 8, 16, 32
                           (per-system form) at [0..4], schedules 0 and 1 (merged) at [5], [6] */
    int merged;
    int schedule;
} fmm_batch_stats_t;
int fmm_batch_get_stats(fmm_batch_t batch, fmm_batch_stats_t *stats);

/*
 * fmm_batch_set_schedule — fixes the merged form's schedule instead of timing
 * both on the next capture: 0 one stream, 1 the near field on a second
 * stream; -1 returns to the autotuner.  The next fmm_batch_eval records and
 * captures its graph again.  Both schedules give the same results bit for
 * bit.  Errors: FMM_ERR_ARG (null batch, another value).
 */
int fmm_batch_set_schedule(fmm_batch_t batch, int schedule);

/*
 * fmm_eval_static — fmm_eval without a workspace argument.  The paper has no
 * counterpart: this entry point is for callers that cannot allocate device
 * memory at the time they evaluate (a plugin inside a host application whose
 * device memory is all owned by the host's allocator or pool, real-time
 * time-step loops that must not allocate, deployments that fix their device
 * memory at start-up).
 *   Scratch: a static device array of FMM_STATIC_WORKSPACE_BYTES (32 MiB),
 *   which every GPU that loads the library holds until the process exits.
 *   Limit: (plan, n) whose fmm_workspace_size exceeds it are rejected with
 *   FMM_ERR_WORKSPACE before any device work.
 *   Allocation: none (no cudaMalloc/cudaFree, no allocating library call);
 *   the plan, created beforehand, owns its tables.
 *   Device: the current device must be the one the plan was created on, else
 *   FMM_ERR_ARG.
 *   Set-up: the first call on a device, with that device current, looks up
 *   the array's device address (cudaGetSymbolAddress).
 *   Status: with opts.sync = 1 the call waits and returns the device status;
 *   with opts.sync = 0, fmm_status(plan, NULL, stream) reads it later.
 *   Sharing: every call uses the same array and leaves the last call's
 *   contents in it (the call clears what must start at zero itself); calls
 *   that overlap on the GPU (other streams, other host threads) race and
 *   must be serialised by the caller.
 * Arguments and results as fmm_eval.
 */
#define FMM_STATIC_WORKSPACE_BYTES (32u << 20)
int fmm_eval_static(fmm_plan_t plan, int64_t n, const float *pos, const float *q,
                    void *potential, double *energy, void *forces, void *stream);

/* Static string naming a status code. */
const char *fmm_strerror(int status);

/* Library version, major*10000 + minor*100 + patch. */
int fmm_version(void);

#ifdef __cplusplus
}
#endif
#endif /* FMM_GB300_H */

// Bilinear forms of the interaction lists (§2.2 step 3, eq. bilinear) on the
// 5th-generation tensor cores (tcgen05): 3-pass split TF32, 1-pass TF32 or
// 3-pass split BF16, FP32 accumulation.
//
// Only cells that hold charges get a functional (step 4 reads no other).
// After the sort, a list of the occupied cells of every (level, target
// parity) segment is built in coarse Morton order; one CTA takes 128 of them
// (the MMA's M).  For each of the 189 interaction-list offsets o, the tile's
// contribution L[cell][a] += sum_b Phi[cell + o][b] K_o[a][b] is a
// 128 x N x K GEMM (N = K = p^3 padded to a multiple of 32): A holds the
// tile's 128 source vectors, B the unit-cell kernel K_o, both in 128-byte K
// chunks staged in shared memory with the 128-byte swizzle; one thread issues
// the MMAs into tensor memory.  A arrives in one of two ways:
//   - box tiles (a segment whose cells mostly hold charges, or a level with
//     fewer than 8 coarse cells per axis): the tile is 128 consecutive
//     Morton cells, an 8 x 4 x 4 box of the padded parity-major layout, and
//     each stage's A is one TMA box copy; one thread issues A and B into the
//     same ring stage;
//   - gathered tiles (sparser segments): producer warps copy each row's 128
//     bytes with 16-byte cp.async straight into the swizzled layout, complete
//     and fence them for the async proxy before arriving on the stage; B has
//     its own TMA producer and ring (tile widths N >= 128), so several stages
//     of gathered copies stay in flight.
//
// Accuracy.  Split precision: x = hi + lo with hi = x with its 13 low mantissa
// bits cleared (exact in TF32); D = Ahi Bhi + Ahi Blo + Alo Bhi.  The BF16
// form splits x = hi + lo with hi = bf16(x), lo = bf16(x - hi) (both round to
// nearest, 8 + 8 significant bits) and takes the same three products with
// kind::f16 MMAs (K = 16 per MMA, 64 per 128-byte chunk).  The 1-pass TF32
// form takes Ahi Bhi alone.  The kernel
// is split as K_o = Kbar_o[a] + Kt_o[a,b] (row mean): the tensor cores contract
// Kt_o, the CUDA cores add Kbar_o[a] Q (Q = the source cell's total charge).
// Each offset accumulates into a fresh TMEM region (two regions, alternating):
// the epilogue warps read it out and add the 189 partials in FP32 registers,
// so no FP32 accumulator in TMEM sees more than 3 * K / 8 MMAs (the tensor
// cores' accumulation is not round-to-nearest; over 1512 MMAs it drifted by
// ~1e-4).  A row's functional depends on its own A rows only, so it is the
// same, bit for bit, whichever tile form computes it.  For N > 64 the
// epilogue splits the columns over two warp groups.
#include <algorithm>
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include "fmm_internal.cuh"
#include "launch.cuh"
#include "tc_ptx.cuh"

namespace fmm {

#define TC_M 128
#define TC_ABYTES (TC_M * 128)      // 128 rows x 32 fp32 (one K chunk)
#define TC_WAIT_CYCLES (4LL << 30)  // about 2 s of SM clock
#define TC_NOFF 189

// records the first wait of the launch that gave up (diagnostics in the header)
__device__ __forceinline__ void tc_wait_failed(int *status, int site, int level, int iter) {
    WsHeader *h = reinterpret_cast<WsHeader *>(status);
    if (atomicCAS(&h->wait_site, 0, site) == 0) {
        h->wait_block = blockIdx.x;
        h->wait_level = level;
        h->wait_iter = iter;
    }
}

// The i-th offset of the interaction list of parity (bx, by, bz), in the
// order shared by the producer and the epilogue.
struct Off {
    int oi, spar, dX, dY, dZ;
};
__device__ __forceinline__ bool next_offset(int bx, int by, int bz, int &ox, int &oy, int &oz) {
    do {
        if (++ox > 3 - bx) {
            ox = -2 - bx;
            if (++oy > 3 - by) {
                oy = -2 - by;
                if (++oz > 3 - bz) return false;
            }
        }
    } while (ox >= -1 && ox <= 1 && oy >= -1 && oy <= 1 && oz >= -1 && oz <= 1);
    return true;
}
__device__ __forceinline__ Off make_off(int bx, int by, int bz, int ox, int oy, int oz) {
    Off f;
    const int sx = bx + ox, sy = by + oy, sz = bz + oz;
    f.spar = (sx & 1) | ((sy & 1) << 1) | ((sz & 1) << 2);
    f.dX = sx >> 1;
    f.dY = sy >> 1;
    f.dZ = sz >> 1;
    f.oi = ((oz + 3) * 7 + (oy + 3)) * 7 + (ox + 3);
    return f;
}

#define TC_TF32X3 0
#define TC_TF32X1 1
#define TC_BF16X3 2

template <int N, int MODE>
struct TcShape {
    static constexpr int CH = N > 64 ? 2 : 1;           // epilogue column groups
    static constexpr int EPI = 4 * CH;                  // epilogue warps
    static constexpr int KE = MODE == TC_BF16X3 ? 64 : 32;  // K elements per 128-byte chunk
    static constexpr int KC = (N + KE - 1) / KE;        // 128-byte K chunks
    static constexpr bool LO = MODE != TC_TF32X1;       // lo parts loaded and used
    static constexpr int BBYTES = N * 128;              // one K chunk of K_o (hi or lo)
    static constexpr int TCOLS = 2 * N <= 64 ? 64 : (2 * N <= 128 ? 128 : (2 * N <= 256 ? 256 : 512));
    static constexpr int COLS = N / CH;                 // columns per epilogue thread
};

// ---------------------------------------------------------------------------
// Occupied cells.  Only the functionals of cells that hold a charge are read
// (step 4 evaluates a cell's functional at its own charges, and a cell with
// charges has a parent with charges), so the contraction forms those alone:
// its 128-row tiles are cut from a list of the occupied cells of each (level,
// target parity) segment, in coarse Morton order, built after the sort.
// ---------------------------------------------------------------------------
struct OccParams {
    const int *leaf_start;
    int *occ;  // the workspace region (layout in fmm_internal.cuh)
    int depth, lmin, nseg, nblk;
    int N;     // tile width of the contraction (box or gathered tiles per segment)
    int bfirst[8 * (FMM_MAXDEPTH + 1) + 1];  // first block of each segment
};

// block -> segment, level, parity and its first coarse cell
__device__ __forceinline__ int occ_block_segment(const OccParams &op, int bid, int &l, int &par, int64_t &c0) {
    int s = 0;
    while (s + 1 < op.nseg && bid >= op.bfirst[s + 1]) s++;
    l = op.lmin + s / 8;
    par = s & 7;
    c0 = (int64_t)(bid - op.bfirst[s]) * OCC_BLOCK;
    return s;
}

// Occupancy of the four consecutive coarse cells of this thread (bit k: cell
// c0 + 4 threadIdx.x + k) and the block's exclusive prefix of their count.
__device__ __forceinline__ unsigned occ_flags(const OccParams &op, int l, int par, int64_t c0, int &pre,
                                              int &total) {
    __shared__ int wsum[OCC_BLOCK / 4 / 32];
    const int64_t ncs = occ_seg_cells(op.lmin, 8 * (l - op.lmin));
    unsigned f = 0;
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const int64_t kc = c0 + 4 * threadIdx.x + k;
        if (kc < ncs && cell_occupied(op.leaf_start, op.depth, l, kc * 8 + par)) f |= 1u << k;
    }
    const int v = __popc(f), lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) wsum[warp] = inc;
    __syncthreads();
    int before = 0;
    total = 0;
#pragma unroll
    for (int w = 0; w < OCC_BLOCK / 4 / 32; w++) {
        before += w < warp ? wsum[w] : 0;
        total += wsum[w];
    }
    pre = before + inc - v;
    return f;
}

struct KOccCount {
    static constexpr int BS = OCC_BLOCK / 4, MINB = 0;  // bounds on the block size only
    OccParams op;
    __device__ __forceinline__ void run(const int bid_, const int nblk_) const {
        int l, par, pre, total;
        int64_t c0;
        occ_block_segment(op, bid_, l, par, c0);
        occ_flags(op, l, par, c0, pre, total);
        if (threadIdx.x == 0) op.occ[bid_] = total;
    }
};
__global__ void __launch_bounds__(KOccCount::BS) k_occ_count(const __grid_constant__ KOccCount k) {
    k.run(blockIdx.x, gridDim.x);
}

// per segment (one warp each): the blocks' exclusive prefix and the segment's count
struct KOccOffsets {
    static constexpr int BS = 0, MINB = 0;
    OccParams op;
    __device__ __forceinline__ void run(const int bid_, const int nblk_) const {
        int *bcnt = op.occ, *cnt = op.occ + op.nblk;
        const int s = (bid_ * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
        if (s >= op.nseg) return;
        int run = 0;
        for (int b0 = op.bfirst[s]; b0 < op.bfirst[s + 1]; b0 += 32) {
            const int b = b0 + lane;
            const int c = b < op.bfirst[s + 1] ? bcnt[b] : 0;
            int inc = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            if (b < op.bfirst[s + 1]) bcnt[b] = run + inc - c;
            run += __shfl_sync(0xffffffffu, inc, 31);
        }
        if (lane == 0) cnt[s] = run;
    }
};
__global__ void k_occ_offsets(const __grid_constant__ KOccOffsets k) {
    k.run(blockIdx.x, gridDim.x);
}

// the list entries: coarse coordinates X | Y << 10 | Z << 20 of each occupied
// cell; block 0 also writes the prefix of the segments' 128-row tiles
struct KOccScatter {
    static constexpr int BS = OCC_BLOCK / 4, MINB = 0;  // bounds on the block size only
    OccParams op;
    __device__ __forceinline__ void run(const int bid_, const int nblk_) const {
        int l, par, pre, total;
        int64_t c0;
        const int s = occ_block_segment(op, bid_, l, par, c0);
        unsigned f = occ_flags(op, l, par, c0, pre, total);
        int *dst = op.occ + occ_list_offset(op.depth, op.lmin) + occ_seg_first(op.lmin, s) + op.occ[bid_] + pre;
        for (int k = 0; k < 4; k++) {
            if (f & (1u << k)) {
                int X, Y, Z;
                morton_decode((uint32_t)(c0 + 4 * threadIdx.x + k), X, Y, Z);
                *dst++ = X | (Y << 10) | (Z << 20);
            }
        }
        if (bid_ == 0 && threadIdx.x == 0) {
            const int *cnt = op.occ + op.nblk;
            int *tiles = op.occ + op.nblk + op.nseg;
            int t = 0;
            for (int k = 0; k < op.nseg; k++) {
                tiles[k] = t;
                t += occ_seg_tiles(1 << (op.lmin + k / 8 - 1), cnt[k], op.N);
            }
            tiles[op.nseg] = t;
        }
    }
};
__global__ void __launch_bounds__(KOccScatter::BS) k_occ_scatter(const __grid_constant__ KOccScatter k) {
    k.run(blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------------
// The contraction over the occupied-cell lists.  One CTA per 128-row tile of a
// segment (level l, target parity b): row r is the tile's r-th occupied
// target cell; for offset o its A operand row is the source cell (target + o)
// of the operand layout, gathered by the producer warps with 16-byte
// cp.async copies straight into the 128-byte-swizzled K-major layout (the
// 16-byte chunk j of row r lands at chunk j ^ (r mod 8)); the kernel matrix B
// arrives by TMA as in the box form.  The copies of a stage are complete and
// fenced for the async proxy before the producers arrive on its barrier.  MMA
// issue, TMEM regions and the epilogue are those of the box form, so every
// row is summed over the offsets in the same order: a row's functional is the
// box form's bit for bit.
// ---------------------------------------------------------------------------
struct TcgParams {
    CUtensorMap k_hi, k_lo;
    CUtensorMap phi_hi[FMM_MAXDEPTH + 1], phi_lo[FMM_MAXDEPTH + 1];  // box maps of the operand layout
    const char *op_hi, *op_lo;  // operand copies of the grid charges (every level)
    int row_bytes;              // bytes of one cell vector in the operand layout
    int lmin, depth, p3, spow, nseg;
    const int *occ;             // occupied-cell lists
    long long op_cell0[FMM_MAXDEPTH + 2];  // first operand cell of each level
    long long loc_off[FMM_MAXDEPTH + 1];
    long long q_off[FMM_MAXDEPTH + 1];
    float *loc;
    const float *qlev;
    const float *kbar;  // [343][N], zero padded
    int *status;
    int inject_stall;   // test hook: the first stage's kernel copies are withheld
    // Cross-system tiles (batched evaluations; xsys != nullptr): the levels
    // lmin..depth of many systems whose levels have fewer than 8 coarse cells
    // per axis, every cell of every system one row, gathered.  xseg: [nseg]
    // rows per segment, [nseg + 1] prefix of their tiles, [nseg] first list
    // entry, then the list (system << 12 | Z << 8 | Y << 4 | X); xsys: per
    // system its operand copies, charges and functionals (op_hi, op_lo, qlev,
    // loc above are unused).
    const TcXSys *xsys;
    const int *xseg;
};

// Ring depths per tile shape.  N >= 128: the gathered A stages (32 KB each)
// and the kernel-matrix B stages (2 N 128 bytes) are separate rings with their
// own producers, so the gather keeps G = SA - 1 stages of copies in flight per
// producer thread; one CTA per SM (N = 224: 3 A + 2 B stages, 208 KB; N = 128:
// 3 + 3, 192 KB).  Dynamic plus static shared memory stays below 227 KB.  N <= 64 (UNI): one ring whose stages hold A and B, one
// producer warp whose first lane also issues the B copies, six warps and two
// CTAs per SM (each CTA's barrier round trips and epilogue hide under the
// other's MMAs).
template <int N, int MODE, bool CROSS = false>
struct TcgShape {
    typedef TcShape<N, MODE> B;
    static constexpr bool UNI = N <= 64;
    // producer (gather) warps: cross-system tiles of the narrow shapes gather
    // every row (no box copies), with two warps
    static constexpr int PW = UNI ? (CROSS ? 2 : 1) : 2;
    static_assert(32 % PW == 0, "the gather's row groups: 32 per stage, PW warps");
    static constexpr int NPROD = 32 * PW;
    static constexpr int SA = UNI ? 2 : 3;
    static constexpr int SB = N == 128 ? 3 : 2;
    static constexpr int G = SA - 1;                 // copy groups in flight per producer thread
    static constexpr int ASTAGE = 2 * TC_ABYTES;     // hi, lo
    static constexpr int BSTAGE = 2 * B::BBYTES;     // hi, lo
    static constexpr int WB = B::EPI + PW;           // kernel-matrix TMA warp (split rings)
    static constexpr int WM = UNI ? WB : WB + 1;     // MMA warp
    static constexpr int THREADS = 32 * (WM + 1);
    static constexpr int MINB = UNI ? 2 : 1;
    // rings, barriers, the rows' tables (cross-system tiles: also each row's
    // system and its operand addresses)
    static constexpr int SMEM = 1024 + SA * ASTAGE + SB * BSTAGE + 256 + 3 * TC_M * 4 + (CROSS ? TC_M * 4 + 2 * TC_M * 8 : 0);
    static_assert(SMEM + 1024 <= 227 * 1024, "shared memory of one CTA");
};

template <int G>
__device__ __forceinline__ void cp_async_wait_pending() {
    asm volatile("cp.async.wait_group %0;" ::"n"(G) : "memory");
}

template <int N, int MODE, bool CROSS = false>
struct KM2LTcg {
    static constexpr int BS = TcgShape<N, MODE, CROSS>::THREADS, MINB = TcgShape<N, MODE, CROSS>::MINB;
    static constexpr int SMEM = TcgShape<N, MODE, CROSS>::SMEM;
    TcgParams prm;
    __device__ __forceinline__ void run(const int bid_, const int nblk_) const {
        typedef TcShape<N, MODE> Sh;
        typedef TcgShape<N, MODE, CROSS> Gh;
        // the segments' counts and tile prefix, read once into shared memory
        __shared__ int seg_cnt[8 * (FMM_MAXDEPTH + 1)], seg_tiles[8 * (FMM_MAXDEPTH + 1) + 1];
        constexpr bool cross = CROSS;
        {
            const int *cnt_g = cross ? prm.xseg : prm.occ + occ_nblk(prm.depth, prm.lmin), *tiles_g = cnt_g + prm.nseg;
            if ((int)threadIdx.x <= prm.nseg) seg_tiles[threadIdx.x] = tiles_g[threadIdx.x];
            if ((int)threadIdx.x < prm.nseg) seg_cnt[threadIdx.x] = cnt_g[threadIdx.x];
            __syncthreads();
        }
        if ((int)bid_ >= seg_tiles[prm.nseg]) return;  // past the last occupied tile
        int sg = 0;
        while (sg + 1 < prm.nseg && (int)bid_ >= seg_tiles[sg + 1]) sg++;
        const int l = prm.lmin + sg / 8, par = sg & 7;
        const int bx = par & 1, by = (par >> 1) & 1, bz = par >> 2;
        const int H = 1 << (l - 1), P = H + 2, Pt = (int)tc_level_extent(l);
        const int count = seg_cnt[sg];
        const int r0 = ((int)bid_ - seg_tiles[sg]) * TC_M;  // first list entry of the tile
        const int *lst = cross ? prm.xseg + 3 * prm.nseg + 1 + prm.xseg[2 * prm.nseg + 1 + sg]
                               : prm.occ + occ_list_offset(prm.depth, prm.lmin) + occ_seg_first(prm.lmin, sg);

        extern __shared__ unsigned char smraw[];
        const uint32_t raw = tc::smem_u32(smraw);
        const uint32_t abase = (raw + 1023u) & ~1023u;           // A ring
        const uint32_t bbase = abase + Gh::SA * Gh::ASTAGE;       // B ring
        const uint32_t bars = bbase + Gh::SB * Gh::BSTAGE;
        const uint32_t afull0 = bars, aempty0 = afull0 + 8 * Gh::SA;
        const uint32_t bfull0 = aempty0 + 8 * Gh::SA, bempty0 = bfull0 + 8 * Gh::SB;
        const uint32_t rfull0 = bempty0 + 8 * Gh::SB, rfree0 = rfull0 + 16;
        const uint32_t done = rfree0 + 16;
        const uint32_t tslot = done + 8;
        volatile uint32_t *tslot_ptr = reinterpret_cast<volatile uint32_t *>(smraw + (tslot - raw));
        // per row: source-cell base in the operand layout, cell in the padded
        // Phi layout (charges Q), target cell in the L layout (-1: past the
        // list); cross-system tiles: its system and the addresses of its source
        // cell in that system's hi / lo operand copies
        int *rowA = reinterpret_cast<int *>(smraw + (bars - raw) + 256);
        int *rowQ = rowA + TC_M, *rowL = rowQ + TC_M, *rowS = rowL + TC_M;
        const char **rowBh = reinterpret_cast<const char **>(rowS + TC_M), **rowBl = rowBh + TC_M;

        // Box tiles (occ_box_segment: a level with fewer than 8 coarse cells per
        // axis, or a segment whose cells mostly hold charges): tile t is the 128
        // consecutive Morton cells [128 t, 128 t + 128), one 8 x 4 x 4 box, and
        // each offset's A operand is one TMA box copy (row r = x + 8 y + 32 z of
        // the box) instead of 128 gathered rows.  A level with fewer than 8 coarse
        // cells per axis takes one box at the origin, partly outside the grid (the
        // operand layout holds zeros there; those rows are not stored).
        const bool box = !cross && occ_box_segment(H, count, N);
        // one ring whose stages hold A and B, filled by one thread (box tiles, and
        // every tile of the narrow shapes), or split rings (gathered tiles of N >= 128)
        const bool uni = Gh::UNI || box;
        const int SU = Gh::SA < Gh::SB ? Gh::SA : Gh::SB;
        const int ra = uni ? SU : Gh::SA, rb = uni ? SU : Gh::SB;  // ring depths of A and B
        int X0 = 0, Y0 = 0, Z0 = 0;
        if (box) morton_decode((uint32_t)r0, X0, Y0, Z0);
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        if (threadIdx.x < TC_M) {
            const int r = threadIdx.x;
            int X, Y, Z;
            bool in;
            if (box) {
                X = X0 + (r & 7);
                Y = Y0 + ((r >> 3) & 3);
                Z = Z0 + (r >> 5);
                in = X < H && Y < H && Z < H;
            } else {
                in = r0 + r < count;
                const int pk = lst[in ? r0 + r : r0];  // rows past the list repeat the tile's first cell
                if (cross) {
                    X = pk & 15;
                    Y = (pk >> 4) & 15;
                    Z = (pk >> 8) & 15;
                    rowS[r] = pk >> 12;
                } else {
                    X = pk & 1023;
                    Y = (pk >> 10) & 1023;
                    Z = pk >> 20;
                }
            }
            rowA[r] = ((Z + 1) * Pt + Y + 1) * Pt + X + 1;
            rowQ[r] = ((Z + 1) * P + Y + 1) * P + X + 1;
            rowL[r] = in ? ((par * H + Z) * H + Y) * H + X : -1;
            if (cross) {
                const TcXSys &xs = prm.xsys[rowS[r]];
                rowBh[r] = xs.op_hi + (int64_t)rowA[r] * prm.row_bytes;
                rowBl[r] = xs.op_lo + (int64_t)rowA[r] * prm.row_bytes;
            }
        }
        if (threadIdx.x == 0) {
            for (int s = 0; s < Gh::SA; s++) {
                // arrivals: the box copies' issuer, or every gather thread (plus the
                // issuer of the B copies when they share the ring)
                tc::mbar_init(afull0 + 8 * s, box ? 1 : Gh::NPROD + (uni ? 1 : 0));
                tc::mbar_init(aempty0 + 8 * s, 1);
            }
            for (int s = 0; s < Gh::SB; s++) {
                tc::mbar_init(bfull0 + 8 * s, 1);
                tc::mbar_init(bempty0 + 8 * s, 1);
            }
            for (int r = 0; r < 2; r++) {
                tc::mbar_init(rfull0 + 8 * r, 1);
                tc::mbar_init(rfree0 + 8 * r, 32 * Sh::EPI);
            }
            tc::mbar_init(done, 1);
            tc::fence_barrier_init();
        }
        if (warp == 0) tc::tmem_alloc(tslot, Sh::TCOLS);
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        const uint32_t tmem = *tslot_ptr;

        if (warp >= Sh::EPI && warp < Sh::EPI + Gh::PW && (!box || (warp == Sh::EPI && lane == 0))) {
            // ---- A producers.  Box tiles: the first lane issues one TMA box (hi,
            //      lo) per stage.  Otherwise the gather: lane = (row within a group
            //      of four) * 8 + 16-byte chunk, warp pw takes rows 4 (pw + PW i) +
            //      lane / 8; a stage is signalled once its copies are complete and
            //      fenced for the async proxy, G - 1 stages later (G stages of copies
            //      in flight).  With one ring (UNI) the first lane also issues the
            //      stage's B copies. ----
            const int pw = warp - Sh::EPI;
            const bool lead = pw == 0 && lane == 0;
            if (lead) {
                if (box) {
                    tc::tensormap_acquire(&prm.phi_hi[l]);
                    if (Sh::LO) tc::tensormap_acquire(&prm.phi_lo[l]);
                }
                if (uni) {
                    tc::tensormap_acquire(&prm.k_hi);
                    if (Sh::LO) tc::tensormap_acquire(&prm.k_lo);
                }
            }
            const int j = lane & 7, rsub = lane >> 3;
            constexpr uint32_t ABYTES = Sh::LO ? 2 * TC_ABYTES : TC_ABYTES;
            constexpr uint32_t BBYTES = Sh::LO ? 2 * Sh::BBYTES : Sh::BBYTES;
            bool failed = false;
            int last_phase[8] = {-1, -1, -1, -1, -1, -1, -1, -1};
            int sig = 0;  // next gathered stage to signal
            const int64_t lvl0 = prm.op_cell0[l];
            const int64_t pt3 = (int64_t)Pt * Pt * Pt;
            int ox = -2 - bx - 1, oy = -2 - by, oz = -2 - bz, it = 0;
            while (!failed && next_offset(bx, by, bz, ox, oy, oz)) {
                const Off f = make_off(bx, by, bz, ox, oy, oz);
                const int64_t delta = lvl0 + f.spar * pt3 + ((int64_t)f.dZ * Pt + f.dY) * Pt + f.dX;
                const int cX = X0 + 1 + f.dX, cY = Y0 + 1 + f.dY, cZ = Z0 + 1 + f.dZ;
                for (int kc = 0; kc < Sh::KC; kc++, it++) {
                    const int s = it % ra;
                    const uint32_t ph = (uint32_t)(it / ra) & 1u;
                    if (!tc::mbar_wait(aempty0 + 8 * s, ph ^ 1u, TC_WAIT_CYCLES)) {
                        if (lane == 0) tc_wait_failed(prm.status, 1, l, it);
                        failed = true;
                        break;
                    }
                    const uint32_t st = abase + s * Gh::ASTAGE;
                    const uint32_t fb = afull0 + 8 * s;
                    // TMA bytes of this stage (an arrival of its own; none when the
                    // lead only gathers)
                    const uint32_t tx = (box ? ABYTES : 0u) + (uni ? BBYTES : 0u);
                    if (lead && tx) {
                        tc::mbar_expect_tx(fb, tx);
                        last_phase[s] = (int)ph;
                        if (box) {
                            tc::tma_load_5d(st, &prm.phi_hi[l], fb, kc * Sh::KE, cX, cY, cZ, f.spar);
                            if (Sh::LO) tc::tma_load_5d(st + TC_ABYTES, &prm.phi_lo[l], fb, kc * Sh::KE, cX, cY, cZ, f.spar);
                        }
                        if (uni && !(prm.inject_stall && it == 0)) {  // inject: armed, never filled
                            const uint32_t stb = bbase + s * Gh::BSTAGE;
                            tc::tma_load_3d(stb, &prm.k_hi, fb, kc * Sh::KE, 0, f.oi);
                            if (Sh::LO) tc::tma_load_3d(stb + Sh::BBYTES, &prm.k_lo, fb, kc * Sh::KE, 0, f.oi);
                        }
                    }
                    if (box) continue;
                    const int64_t cb = (int64_t)kc * 128 + j * 16;
                    if (cross) {  // each row from its system's operand copies
                        const int64_t src = delta * prm.row_bytes + cb;
#pragma unroll 4
                        for (int i = 0; i < 32 / Gh::PW; i++) {
                            const int r = 4 * (pw + Gh::PW * i) + rsub;
                            const uint32_t d = st + r * 128 + ((j ^ (r & 7)) << 4);
                            tc::cp_async16(d, rowBh[r] + src);
                            if (Sh::LO) tc::cp_async16(d + TC_ABYTES, rowBl[r] + src);
                        }
                    } else {
#pragma unroll 4
                        for (int i = 0; i < 32 / Gh::PW; i++) {
                            const int r = 4 * (pw + Gh::PW * i) + rsub;
                            const int64_t src = (delta + rowA[r]) * prm.row_bytes + cb;
                            const uint32_t d = st + r * 128 + ((j ^ (r & 7)) << 4);
                            tc::cp_async16(d, prm.op_hi + src);
                            if (Sh::LO) tc::cp_async16(d + TC_ABYTES, prm.op_lo + src);
                        }
                    }
                    tc::cp_async_commit();
                    cp_async_wait_pending<Gh::G - 1>();  // stages <= it - G + 1 have landed
                    if (it - Gh::G + 1 >= sig) {
                        tc::fence_proxy_async_smem();
                        for (; sig <= it - Gh::G + 1; sig++) tc::mbar_arrive(afull0 + 8 * (sig % ra));
                    }
                }
            }
            if (!box) {
                tc::cp_async_wait_all();  // no copy outlives the CTA
                if (!failed) {
                    tc::fence_proxy_async_smem();
                    for (; sig < it; sig++) tc::mbar_arrive(afull0 + 8 * (sig % ra));
                }
            }
            if (failed) {
                if (lane == 0) atomicOr(prm.status, ST_TIMEOUT);
                if (lead)  // the TMA copies already issued land before the CTA can exit
                    for (int s = 0; s < ra; s++)
                        if (last_phase[s] >= 0) tc::mbar_wait(afull0 + 8 * s, (uint32_t)last_phase[s], TC_WAIT_CYCLES);
            }
        } else if (!uni && warp == Gh::WB && lane == 0) {
            tc::tensormap_acquire(&prm.k_hi);
            if (Sh::LO) tc::tensormap_acquire(&prm.k_lo);
            // ---- kernel-matrix producer (split rings): K chunk kc of K_o by TMA ----
            bool failed = false;
            int last_phase[4] = {-1, -1, -1, -1};
            int ox = -2 - bx - 1, oy = -2 - by, oz = -2 - bz, it = 0;
            while (!failed && next_offset(bx, by, bz, ox, oy, oz)) {
                const Off f = make_off(bx, by, bz, ox, oy, oz);
                for (int kc = 0; kc < Sh::KC; kc++, it++) {
                    const int s = it % Gh::SB;
                    const uint32_t ph = (uint32_t)(it / Gh::SB) & 1u;
                    if (!tc::mbar_wait(bempty0 + 8 * s, ph ^ 1u, TC_WAIT_CYCLES)) {
                        tc_wait_failed(prm.status, 1, l, it);
                        failed = true;
                        break;
                    }
                    const uint32_t st = bbase + s * Gh::BSTAGE;
                    const uint32_t fb = bfull0 + 8 * s;
                    tc::mbar_expect_tx(fb, Sh::LO ? 2 * Sh::BBYTES : Sh::BBYTES);
                    last_phase[s] = (int)ph;
                    if (prm.inject_stall && it == 0) continue;  // armed, never filled (test hook)
                    tc::tma_load_3d(st, &prm.k_hi, fb, kc * Sh::KE, 0, f.oi);
                    if (Sh::LO) tc::tma_load_3d(st + Sh::BBYTES, &prm.k_lo, fb, kc * Sh::KE, 0, f.oi);
                }
            }
            if (failed) {
                atomicOr(prm.status, ST_TIMEOUT);
                // the copies already issued land before the CTA can exit
                for (int s = 0; s < Gh::SB; s++)
                    if (last_phase[s] >= 0) tc::mbar_wait(bfull0 + 8 * s, (uint32_t)last_phase[s], TC_WAIT_CYCLES);
            }
        } else if (warp == Gh::WM && lane == 0) {
            // ---- MMA issuer: offset i accumulates into TMEM region i & 1 ----
            const uint32_t idesc = MODE == TC_BF16X3 ? tc::idesc_bf16(TC_M, N) : tc::idesc_tf32(TC_M, N);
            bool failed = false;
            for (int i = 0; i < TC_NOFF && !failed; i++) {
                const int r = i & 1;
                const uint32_t u = (uint32_t)(i >> 1) & 1u;
                if (!tc::mbar_wait(rfree0 + 8 * r, u ^ 1u, TC_WAIT_CYCLES)) {
                    tc_wait_failed(prm.status, 2, l, i);
                    failed = true;
                    break;
                }
                const uint32_t d = tmem + (uint32_t)(r * N);
                for (int kc = 0; kc < Sh::KC; kc++) {
                    const int it = Sh::KC * i + kc;
                    const int sa = it % ra, sb = it % rb;
                    if (!tc::mbar_wait(afull0 + 8 * sa, (uint32_t)(it / ra) & 1u, TC_WAIT_CYCLES) ||
                        (!uni && !tc::mbar_wait(bfull0 + 8 * sb, (uint32_t)(it / rb) & 1u, TC_WAIT_CYCLES))) {
                        tc_wait_failed(prm.status, 3, l, it);
                        failed = true;
                        break;
                    }
                    tc::fence_after_sync();
                    const uint32_t sta = abase + sa * Gh::ASTAGE, stb = bbase + sb * Gh::BSTAGE;
#pragma unroll
                    for (int k = 0; k < 4; k++) {  // 32 bytes of K per MMA (8 tf32 or 16 bf16)
                        const uint64_t ah = tc::desc_sw128(sta + 32 * k);
                        const uint64_t al = tc::desc_sw128(sta + TC_ABYTES + 32 * k);
                        const uint64_t bh = tc::desc_sw128(stb + 32 * k);
                        const uint64_t bl = tc::desc_sw128(stb + Sh::BBYTES + 32 * k);
                        if (MODE == TC_BF16X3) {
                            tc::mma_bf16(d, ah, bh, idesc, (kc | k) != 0);
                            tc::mma_bf16(d, ah, bl, idesc, 1u);
                            tc::mma_bf16(d, al, bh, idesc, 1u);
                        } else {
                            tc::mma_tf32(d, ah, bh, idesc, (kc | k) != 0);
                            if (MODE == TC_TF32X3) {
                                tc::mma_tf32(d, ah, bl, idesc, 1u);
                                tc::mma_tf32(d, al, bh, idesc, 1u);
                            }
                        }
                    }
                    tc::mma_commit(aempty0 + 8 * sa);
                    if (!uni) tc::mma_commit(bempty0 + 8 * sb);
                }
                if (!failed) tc::mma_commit(rfull0 + 8 * r);
            }
            if (failed) atomicOr(prm.status, ST_TIMEOUT);
            tc::mma_commit(done);  // always: the deallocation waits on it
        } else if (warp < Sh::EPI) {
            // ---- epilogue: TMEM lane = row; columns [c0, c0 + COLS) ----
            const int sub = warp & 3, cgrp = warp >> 2;
            const int c0 = cgrp * Sh::COLS;
            const int row = sub * 32 + lane;
            const int lrow = rowL[row];
            const bool valid = lrow >= 0;
            const float *q = (cross ? prm.xsys[rowS[row]].qlev : prm.qlev) + prm.q_off[l] + rowQ[row];
            const int64_t pp3 = (int64_t)P * P * P;
            float tot[Sh::COLS];
#pragma unroll
            for (int j = 0; j < Sh::COLS; j++) tot[j] = 0.0f;
            bool ok = true;
            int ox = -2 - bx - 1, oy = -2 - by, oz = -2 - bz;
            for (int i = 0; i < TC_NOFF; i++) {
                next_offset(bx, by, bz, ox, oy, oz);
                const Off f = make_off(bx, by, bz, ox, oy, oz);
                const float Qs = valid ? q[f.spar * pp3 + ((int64_t)f.dZ * P + f.dY) * P + f.dX] : 0.0f;
                const float4 *kb = reinterpret_cast<const float4 *>(prm.kbar + (int64_t)f.oi * N + c0);
                const int r = i & 1;
                const uint32_t u = (uint32_t)(i >> 1) & 1u;
                if (ok && !tc::mbar_wait(rfull0 + 8 * r, u, TC_WAIT_CYCLES)) {
                    if (lane == 0) tc_wait_failed(prm.status, 4, l, i);
                    ok = false;
                }
                tc::fence_after_sync();
                const uint32_t taddr = tmem + ((uint32_t)(sub * 32) << 16) + (uint32_t)(r * N + c0);
#pragma unroll
                for (int c = 0; c < Sh::COLS / 16; c++) {
                    uint32_t v[16];
                    tc::tmem_ld16(taddr + c * 16, v);
#pragma unroll
                    for (int j = 0; j < 16; j += 4) {
                        const float4 m = kb[(c * 16 + j) >> 2];
                        tot[c * 16 + j] += __uint_as_float(v[j]) + m.x * Qs;
                        tot[c * 16 + j + 1] += __uint_as_float(v[j + 1]) + m.y * Qs;
                        tot[c * 16 + j + 2] += __uint_as_float(v[j + 2]) + m.z * Qs;
                        tot[c * 16 + j + 3] += __uint_as_float(v[j + 3]) + m.w * Qs;
                    }
                }
                tc::fence_before_sync();
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(rfree0 + 8 * r) : "memory");
            }
            const int p3 = prm.p3;
            float *out = (cross ? prm.xsys[rowS[row]].loc : prm.loc) + prm.loc_off[l] + (int64_t)(valid ? lrow : 0) * p3 + c0;
            const float scale = (float)(1 << (l * prm.spow));
            if (ok) {
                if (valid) {
#pragma unroll
                    for (int j = 0; j < Sh::COLS; j++)
                        if (c0 + j < p3) out[j] = scale * tot[j];
                }
            } else if (lane == 0) {
                atomicOr(prm.status, ST_TIMEOUT);
            }
        }
        tc::fence_before_sync();
        __syncthreads();
        if (warp == 0) {
            tc::mbar_wait(done, 0, TC_WAIT_CYCLES);
            tc::fence_after_sync();
            tc::tmem_dealloc(tmem, Sh::TCOLS);
        }
    }
};
template <int N, int MODE>
__global__ void __launch_bounds__(KM2LTcg<N, MODE>::BS, KM2LTcg<N, MODE>::MINB) k_m2l_tcg(const __grid_constant__ KM2LTcg<N, MODE> k) {
    k.run(blockIdx.x, gridDim.x);
}
// cross-system tiles: launched merged only (their functor lives in the batch's table)
template <int N, int MODE>
__global__ void __launch_bounds__(KM2LTcg<N, MODE, true>::BS, KM2LTcg<N, MODE, true>::MINB)
    k_m2l_tcx(const __grid_constant__ KM2LTcg<N, MODE, true> k) {
    k.run(blockIdx.x, gridDim.x);
}

// Levels lmin..lmax of the grid charges, remapped from the padded layout (P =
// H + 2 per axis) into the operand layout (tc_level_extent per axis, zeros
// outside) and split into hi / lo parts.  One element = one (cell, b) of the
// operand layout.
struct SplitLevels {
    int lmin, lmax;
    long long src[FMM_MAXDEPTH + 2];  // first value of level l in the padded layout
    long long dst[FMM_MAXDEPTH + 2];  // first cell of level l in the operand layout
    long long cst[FMM_MAXDEPTH + 2];  // first visited cell of level l (from lmin; see split_cell)
};
__device__ __forceinline__ bool split_source(const SplitLevels &L, int64_t c, int &l, int64_t &src_cell) {
    l = L.lmin;
    while (l < L.lmax && c >= L.dst[l + 1]) l++;
    const int r = (int)(c - L.dst[l]);  // < 8 * 130^3
    const int Pt = (int)tc_level_extent(l), P = (1 << (l - 1)) + 2;
    if (Pt == P) {  // levels with at least 8 coarse cells per axis: same layout
        src_cell = r;
        return true;
    }
    const int x = r % Pt, y = (r / Pt) % Pt, z = (r / (Pt * Pt)) % Pt, par = r / (Pt * Pt * Pt);
    if (x >= P || y >= P || z >= P) return false;
    src_cell = ((int64_t)(par * P + z) * P + y) * P + x;
    return true;
}

// TF32: hi = x with the 13 low mantissa bits cleared (exact in TF32), lo = x - hi;
// with `nearest` (the 1-pass form, which has no lo term) hi is x rounded to the
// nearest TF32 value (ties away from zero) instead of truncated.  One thread per
// 4 consecutive values of a cell (p3s % 32 == 0).
// Visited cell k -> level l, operand cell c and padded-layout cell src_cell;
// false: c lies outside the padded layout (written as zeros).  Levels below
// lpad visit the padded layout's cells only (no box copy reads the rest of
// their operand layout); the others every operand cell.
__device__ __forceinline__ bool split_cell(const SplitLevels &L, int lpad, int64_t k, int &l, int64_t &c,
                                           int64_t &src_cell) {
    l = L.lmin;
    while (l < L.lmax && k >= L.cst[l + 1]) l++;
    const int64_t r = k - L.cst[l];
    if (l < lpad) {
        const int Pt = (int)tc_level_extent(l), P = (1 << (l - 1)) + 2;
        const int x = (int)(r % P), y = (int)((r / P) % P), z = (int)((r / (P * P)) % P), par = (int)(r / (P * P * P));
        c = L.dst[l] + ((int64_t)(par * Pt + z) * Pt + y) * Pt + x;
        src_cell = r;
        return true;
    }
    c = L.dst[l] + r;
    int l2;
    return split_source(L, c, l2, src_cell);
}

struct KSplitTf32 {
    static constexpr int BS = 0, MINB = 0;
    const float *__restrict__ phi;
    SplitLevels L;
    float *__restrict__ hi;
    float *__restrict__ lo;
    int p3;
    int p3s;
    int nearest;
    int lpad;  // levels below lpad: cells outside the padded layout are not visited (no box reads them)
    __device__ __forceinline__ void run(const int bid_, const int nblk_) const {
        const int q4 = p3s / 4;
        const int64_t n = L.cst[L.lmax + 1] * q4;
        for (int64_t i = bid_ * (int64_t)blockDim.x + threadIdx.x; i < n;
             i += (int64_t)nblk_ * blockDim.x) {
            const int b0 = (int)(i % q4) * 4;
            int l;
            int64_t c, sc;
            const bool in = split_cell(L, lpad, i / q4, l, c, sc);
            const float *src = phi + L.src[l] + sc * p3;
            float v[4], h[4], w[4];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                v[j] = (in && b0 + j < p3) ? src[b0 + j] : 0.0f;
                const uint32_t u = __float_as_uint(v[j]) + (nearest ? 0x1000u : 0u);
                h[j] = __uint_as_float(u & 0xFFFFE000u);
                w[j] = v[j] - h[j];
            }
            *reinterpret_cast<float4 *>(hi + c * p3s + b0) = make_float4(h[0], h[1], h[2], h[3]);
            *reinterpret_cast<float4 *>(lo + c * p3s + b0) = make_float4(w[0], w[1], w[2], w[3]);
        }
    }
};
__global__ void k_split_tf32(const __grid_constant__ KSplitTf32 k) {
    k.run(blockIdx.x, gridDim.x);
}

// BF16: hi = bf16(x), lo = bf16(x - hi), both rounded to nearest even; cell
// vectors of p3k values (zero padded, p3k % 64 == 0).  One thread per 4 values.
struct KSplitBf16 {
    static constexpr int BS = 0, MINB = 0;
    const float *__restrict__ phi;
    SplitLevels L;
    __nv_bfloat16 *__restrict__ hi;
    __nv_bfloat16 *__restrict__ lo;
    int p3;
    int p3k;
    int lpad;  // as KSplitTf32
    __device__ __forceinline__ void run(const int bid_, const int nblk_) const {
        const int q4 = p3k / 4;
        const int64_t n = L.cst[L.lmax + 1] * q4;
        for (int64_t i = bid_ * (int64_t)blockDim.x + threadIdx.x; i < n;
             i += (int64_t)nblk_ * blockDim.x) {
            const int b0 = (int)(i % q4) * 4;
            int l;
            int64_t c, sc;
            const bool in = split_cell(L, lpad, i / q4, l, c, sc);
            const float *src = phi + L.src[l] + sc * p3;
            __nv_bfloat16 h[4], w[4];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                const float v = (in && b0 + j < p3) ? src[b0 + j] : 0.0f;
                h[j] = __float2bfloat16_rn(v);
                w[j] = __float2bfloat16_rn(v - __bfloat162float(h[j]));
            }
            *reinterpret_cast<uint2 *>(hi + c * p3k + b0) = *reinterpret_cast<const uint2 *>(h);
            *reinterpret_cast<uint2 *>(lo + c * p3k + b0) = *reinterpret_cast<const uint2 *>(w);
        }
    }
};
__global__ void k_split_bf16(const __grid_constant__ KSplitBf16 k) {
    k.run(blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

int tc_padded(int p3) { return (p3 + 31) / 32 * 32; }
int tc_padded_k(int p3, int mode) {
    return mode == FMM_TC_BF16X3 ? (p3 + 63) / 64 * 64 : tc_padded(p3);
}

// Grid-charge box map of level l (operand layout): dims (pk b, Pt x, Pt y, Pt z,
// 8 parity), box (one 128-byte chunk of b, 8, 4, 4, 1); fp32 (pk = p3s) or bf16
// (pk = p3k) elements.  Every box the kernel loads lies inside the map.
static int encode_phi_map(CUtensorMap *m, const void *base, int l, int pk, bool bf16) {
    auto enc = encode_fn();
    if (!enc) return FMM_ERR_CUDA;
    const cuuint64_t es_b = bf16 ? 2 : 4;
    const cuuint64_t P = (cuuint64_t)tc_level_extent(l), rb = (cuuint64_t)pk * es_b;
    cuuint64_t dims[5] = {(cuuint64_t)pk, P, P, P, 8};
    cuuint64_t strides[4] = {rb, rb * P, rb * P * P, rb * P * P * P};
    cuuint32_t box[5] = {(cuuint32_t)(128 / es_b), 8, 4, 4, 1};
    cuuint32_t es[5] = {1, 1, 1, 1, 1};
    CUresult r = enc(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5,
                     (void *)base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? FMM_OK : FMM_ERR_CUDA;
}

// Kernel-table map: dims (pk b, p3s a, 343 offsets), box (one 128-byte chunk of b,
// p3s, 1); fp32 tables have pk = p3s, bf16 tables pk = p3k.
int tc_encode_kernel_map(void *map, const void *base, int p3s, int pk, int mode) {
    auto enc = encode_fn();
    if (!enc) return FMM_ERR_CUDA;
    const bool bf16 = mode == FMM_TC_BF16X3;
    const cuuint64_t es_b = bf16 ? 2 : 4;
    cuuint64_t dims[3] = {(cuuint64_t)pk, (cuuint64_t)p3s, 343};
    cuuint64_t strides[2] = {(cuuint64_t)pk * es_b, (cuuint64_t)pk * p3s * es_b};
    cuuint32_t box[3] = {(cuuint32_t)(128 / es_b), (cuuint32_t)p3s, 1};
    cuuint32_t es[3] = {1, 1, 1};
    CUresult r = enc((CUtensorMap *)map,
                     bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                     (void *)base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? FMM_OK : FMM_ERR_CUDA;
}

size_t tc_map_bytes() { return sizeof(CUtensorMap); }

template <int N, int MODE>
static int launch_tcg_kernel(const TcgParams &prm, int blocks, int comp, cudaStream_t st, Tracer &tr) {
    typedef TcgShape<N, MODE> Gh;
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(k_m2l_tcg<N, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 Gh::SMEM) != cudaSuccess)
            return FMM_ERR_CUDA;
        kb_set_smem<KM2LTcg<N, MODE>>(Gh::SMEM);
        attr = true;
    }
    launch_k(tr, FMM_TAG(S_M2L_TC, comp), k_m2l_tcg<N, MODE>, KM2LTcg<N, MODE>{prm}, blocks, Gh::THREADS, Gh::SMEM,
             st);
    return FMM_OK;
}

// the record of a cross-system launch (batched evaluations)
template <int N, int MODE>
static int record_tcx(const TcgParams &prm, int blocks, int comp, Tracer &tr) {
    typedef KM2LTcg<N, MODE, true> K;
    kb_set_smem<K>(K::SMEM);
    launch_k(tr, FMM_TAG(S_M2L_TCX, comp), k_m2l_tcx<N, MODE>, K{prm}, blocks, K::BS, K::SMEM, nullptr);
    return FMM_OK;
}
template <int MODE>
static int record_tcx_mode(int p3s, const TcgParams &prm, int blocks, int comp, Tracer &tr) {
    switch (p3s) {
    case 32: return record_tcx<32, MODE>(prm, blocks, comp, tr);
    case 64: return record_tcx<64, MODE>(prm, blocks, comp, tr);
    case 128: return record_tcx<128, MODE>(prm, blocks, comp, tr);
    case 224: return record_tcx<224, MODE>(prm, blocks, comp, tr);
    default: return FMM_ERR_UNSUPPORTED;
    }
}

template <int MODE>
static int launch_tcg_mode(int p3s, const TcgParams &prm, int blocks, int comp, cudaStream_t st, Tracer &tr) {
    switch (p3s) {
    case 32: return launch_tcg_kernel<32, MODE>(prm, blocks, comp, st, tr);
    case 64: return launch_tcg_kernel<64, MODE>(prm, blocks, comp, st, tr);
    case 128: return launch_tcg_kernel<128, MODE>(prm, blocks, comp, st, tr);
    case 224: return launch_tcg_kernel<224, MODE>(prm, blocks, comp, st, tr);
    default: return FMM_ERR_UNSUPPORTED;
    }
}

int launch_m2l_tc(const Geom &g, const Ptrs<float> &P, const WsLayout &W, const void *k_hi_map,
                  const void *k_lo_map, const float *kbar, int lmin, int mode, int inject,
                  float *loc, int spow, bool split, int comp, cudaStream_t st, Tracer &tr) {
    const int depth = g.depth, p3 = g.p3, p3s = tc_padded(p3), pk = tc_padded_k(p3, mode);
    const bool bf16 = mode == FMM_TC_BF16X3;
    // the grid charges of levels lmin..depth in the operand layout, split into
    // hi / lo parts (the bf16 parts are stored in the same buffers, pk <= 2 p3s)
    SplitLevels SL;
    memset(&SL, 0, sizeof(SL));
    SL.lmin = lmin;
    SL.lmax = depth;
    for (int l = 0; l <= depth + 1; l++) {
        SL.src[l] = l <= depth ? W.phi_level[l] : 0;
        SL.dst[l] = tc_level_first(l);
    }
    // a batch whose small levels run as cross-system (gathered) tiles reads
    // none of their padding
    const int lpad = tr.rec ? tr.tc_lbig : 0;
    SL.cst[lmin] = 0;
    for (int l = lmin; l <= depth; l++) {
        const int64_t P = ((int64_t)1 << (l - 1)) + 2;
        SL.cst[l + 1] = SL.cst[l] + (l < lpad ? 8 * P * P * P : SL.dst[l + 1] - SL.dst[l]);
    }
    tr.begin(FMM_STAGE_M2L, st);
    __nv_bfloat16 *hi16 = reinterpret_cast<__nv_bfloat16 *>(P.phihi);
    __nv_bfloat16 *lo16 = reinterpret_cast<__nv_bfloat16 *>(P.philo);
    if (split) {
        // grid-stride over the levels' (cell, 4 values); small systems take a
        // small grid, so that other work keeps the SMs
        const int64_t units = SL.cst[depth + 1] * ((bf16 ? pk : p3s) / 4);
        const int nbs = (int)std::min<int64_t>(152 * 8, std::max<int64_t>(1, (units + 255) / 256));
        if (bf16)
            launch_k(tr, FMM_TAG(S_SPLIT_TC, 0), k_split_bf16, KSplitBf16{P.phi, SL, hi16, lo16, p3, pk, lpad}, nbs,
                     256, 0, st);
        else
            launch_k(tr, FMM_TAG(S_SPLIT_TC, 0), k_split_tf32,
                     KSplitTf32{P.phi, SL, P.phihi, P.philo, p3, p3s, mode == FMM_TC_TF32X1, lpad}, nbs, 256, 0, st);
        tr.count();
    }
    // a batch whose small levels run as cross-system tiles: this system's own
    // launch takes the levels from tr.tc_lbig up
    if (tr.rec && tr.tc_lbig > lmin) {
        lmin = tr.tc_lbig;
        if (depth < lmin) {
            tr.end();
            return FMM_OK;
        }
    }
    // the occupied cells of every (level, parity) segment, once per evaluation
    OccParams op;
    memset(&op, 0, sizeof(op));
    op.leaf_start = P.leaf_start;
    op.occ = P.occ;
    op.depth = depth;
    op.lmin = lmin;
    op.nseg = occ_nseg(depth, lmin);
    op.N = p3s;
    int nb = 0, blocks = 0;
    for (int s = 0; s < op.nseg; s++) {
        op.bfirst[s] = nb;
        nb += (int)((occ_seg_cells(lmin, s) + OCC_BLOCK - 1) / OCC_BLOCK);
        blocks += (int)((occ_seg_cells(lmin, s) + TC_M - 1) / TC_M);  // tiles if every cell holds charges
    }
    op.bfirst[op.nseg] = nb;
    op.nblk = nb;
    if (split) {
        launch_k(tr, FMM_TAG(S_OCC_COUNT, 0), k_occ_count, KOccCount{op}, nb, OCC_BLOCK / 4, 0, st);
        launch_k(tr, FMM_TAG(S_OCC_OFFSETS, 0), k_occ_offsets, KOccOffsets{op}, (op.nseg + 7) / 8, 256, 0, st);
        launch_k(tr, FMM_TAG(S_OCC_SCATTER, 0), k_occ_scatter, KOccScatter{op}, nb, OCC_BLOCK / 4, 0, st);
        tr.count(3);
    }
    TcgParams prm;
    memset(&prm, 0, sizeof(prm));
    memcpy(&prm.k_hi, k_hi_map, sizeof(CUtensorMap));
    memcpy(&prm.k_lo, k_lo_map, sizeof(CUtensorMap));
    const size_t es = bf16 ? 2 : 4;
    prm.op_hi = reinterpret_cast<const char *>(P.phihi);
    prm.op_lo = reinterpret_cast<const char *>(P.philo);
    prm.row_bytes = (int)((bf16 ? pk : p3s) * es);
    prm.lmin = lmin;
    prm.depth = depth;
    prm.p3 = p3;
    prm.spow = spow;
    prm.nseg = op.nseg;
    prm.occ = P.occ;
    for (int l = 0; l <= depth + 1; l++) prm.op_cell0[l] = tc_level_first(l);
    for (int l = lmin; l <= depth; l++) {
        prm.loc_off[l] = W.loc_level[l];
        prm.q_off[l] = W.q_level[l];
        {  // box maps of the operand layout
            const int64_t cl = tc_level_first(l);
            const void *bh = bf16 ? (const void *)(hi16 + cl * pk) : (const void *)(P.phihi + cl * p3s);
            const void *bl = bf16 ? (const void *)(lo16 + cl * pk) : (const void *)(P.philo + cl * p3s);
            int rc = encode_phi_map(&prm.phi_hi[l], bh, l, pk, bf16);
            if (!rc) rc = encode_phi_map(&prm.phi_lo[l], bl, l, pk, bf16);
            if (rc) return rc;
        }
    }
    prm.loc = loc;
    prm.qlev = P.qlev;
    prm.kbar = kbar;
    prm.status = &P.hdr->status;
    prm.inject_stall = inject == FMM_INJECT_TC_STALL;
    prm.xsys = nullptr;
    prm.xseg = nullptr;
    int rc = mode == FMM_TC_BF16X3   ? launch_tcg_mode<TC_BF16X3>(p3s, prm, blocks, comp, st, tr)
             : mode == FMM_TC_TF32X1 ? launch_tcg_mode<TC_TF32X1>(p3s, prm, blocks, comp, st, tr)
                                     : launch_tcg_mode<TC_TF32X3>(p3s, prm, blocks, comp, st, tr);
    tr.count();
    tr.end();
    return rc;
}

int tc_cross_records(const std::vector<TcXSys> &sys, const std::vector<int> &depth, int ncomp, int lmin,
                     int lmax, int p3, int mode, int spow0, const void *const *k_hi_maps,
                     const void *const *k_lo_maps, const float *const *kbars, const WsLayout &W, int *status,
                     void **dx, size_t *dx_bytes, std::vector<LaunchRec> &out) {
    const int ns = (int)depth.size();
    const int p3s = tc_padded(p3), pk = tc_padded_k(p3, mode);
    const bool bf16 = mode == FMM_TC_BF16X3;
    const int nseg = 8 * (lmax - lmin + 1);
    if (lmax >= 5 || ns >= (1 << 19)) return FMM_ERR_UNSUPPORTED;  // coordinates and systems fit the entries
    // the lists: every cell of every system with that level, system-major
    std::vector<int> cnt(nseg, 0), tiles(nseg + 1, 0), first(nseg, 0), list;
    for (int sg = 0; sg < nseg; sg++) {
        const int l = lmin + sg / 8, par = sg & 7, H = 1 << (l - 1);
        first[sg] = (int)list.size();
        for (int i = 0; i < ns; i++) {
            if (depth[i] < l) continue;
            for (int Z = 0; Z < H; Z++)
                for (int Y = 0; Y < H; Y++)
                    for (int X = 0; X < H; X++) list.push_back(i << 12 | Z << 8 | Y << 4 | X);
        }
        cnt[sg] = (int)list.size() - first[sg];
        tiles[sg + 1] = tiles[sg] + (cnt[sg] + TC_M - 1) / TC_M;
        (void)par;
    }
    // device buffer: the segment table and list, then the systems' table per component
    std::vector<int> seg;
    seg.insert(seg.end(), cnt.begin(), cnt.end());
    seg.insert(seg.end(), tiles.begin(), tiles.end());
    seg.insert(seg.end(), first.begin(), first.end());
    seg.insert(seg.end(), list.begin(), list.end());
    const size_t seg_bytes = (seg.size() * sizeof(int) + 255) / 256 * 256;
    const size_t need = seg_bytes + sizeof(TcXSys) * sys.size();
    if (need > *dx_bytes) {
        if (*dx) cudaFree(*dx);
        *dx = nullptr;
        *dx_bytes = 0;
        if (cudaMalloc(dx, need) != cudaSuccess) return FMM_ERR_OOM;
        *dx_bytes = need;
    }
    char *d = reinterpret_cast<char *>(*dx);
    if (cudaMemcpy(d, seg.data(), seg.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(d + seg_bytes, sys.data(), sizeof(TcXSys) * sys.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return FMM_ERR_CUDA;
    out.clear();
    for (int c = 0; c < ncomp; c++) {
        TcgParams prm;
        memset(&prm, 0, sizeof(prm));
        memcpy(&prm.k_hi, k_hi_maps[c], sizeof(CUtensorMap));
        memcpy(&prm.k_lo, k_lo_maps[c], sizeof(CUtensorMap));
        prm.row_bytes = (int)((bf16 ? pk : p3s) * (bf16 ? 2 : 4));
        prm.lmin = lmin;
        prm.depth = lmax;
        prm.p3 = p3;
        prm.spow = c == 0 ? spow0 : spow0 + 1;
        prm.nseg = nseg;
        for (int l = 0; l <= lmax + 1; l++) prm.op_cell0[l] = tc_level_first(l);
        for (int l = lmin; l <= lmax; l++) {
            prm.loc_off[l] = W.loc_level[l];
            prm.q_off[l] = W.q_level[l];
        }
        prm.kbar = kbars[c];
        prm.status = status;
        prm.xsys = reinterpret_cast<const TcXSys *>(d + seg_bytes) + (size_t)c * ns;
        prm.xseg = reinterpret_cast<const int *>(d);
        Tracer t;
        std::vector<LaunchRec> one;
        t.rec = &one;
        int rc = mode == FMM_TC_BF16X3   ? record_tcx_mode<TC_BF16X3>(p3s, prm, tiles[nseg], c, t)
                 : mode == FMM_TC_TF32X1 ? record_tcx_mode<TC_TF32X1>(p3s, prm, tiles[nseg], c, t)
                                         : record_tcx_mode<TC_TF32X3>(p3s, prm, tiles[nseg], c, t);
        if (rc) return rc;
        out.push_back(std::move(one[0]));
    }
    return FMM_OK;
}

}  // namespace fmm

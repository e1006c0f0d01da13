// Bilinear forms of the interaction lists (§2.2 step 3, eq. bilinear) on the
// 5th-generation tensor cores (tcgen05): 3-pass split TF32, 1-pass TF32 or
// 3-pass split BF16, FP32 accumulation.
//
// For one level, one target parity and one box of 8x4x4 coarse cells (128
// target cells = the MMA's M; the coarsest levels take one box partly outside
// the grid), every one of the 189 interaction-list offsets o
// contributes L[cell][a] += sum_b Phi[cell + o][b] K_o[a][b]: a 128 x N x K
// GEMM (N = K = p^3 padded to a multiple of 32) whose A operand (the 128
// source vectors) is one rectangular box of the padded parity-major grid-charge
// layout and whose B operand is the unit-cell kernel.  Both arrive by TMA, in
// 128-byte K chunks, into a 2-stage ring; one thread issues the MMAs.
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
// ~1e-4).  For N > 64 the epilogue splits the columns over two warp groups.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include "fmm_internal.cuh"
#include "tc_ptx.cuh"

namespace fmm {

#define TC_M 128
#define TC_STAGES_MAX 3  // stages of the TMA ring (per tile shape, see TcShape::STAGES)
#define TC_ABYTES (TC_M * 128)      // 128 rows x 32 fp32 (one K chunk)
#define TC_WAIT_CYCLES (4LL << 30)  // about 2 s of SM clock
#define TC_NOFF 189

struct TcParams;
// records the first wait of the launch that gave up (diagnostics in the header)
__device__ __forceinline__ void tc_wait_failed(int *status, int site, int level, int iter) {
    WsHeader *h = reinterpret_cast<WsHeader *>(status);
    if (atomicCAS(&h->wait_site, 0, site) == 0) {
        h->wait_block = blockIdx.x;
        h->wait_level = level;
        h->wait_iter = iter;
    }
}

struct TcParams {
    CUtensorMap phi_hi[FMM_MAXDEPTH + 1];
    CUtensorMap phi_lo[FMM_MAXDEPTH + 1];
    CUtensorMap k_hi, k_lo;
    int first_block[FMM_MAXDEPTH + 2];
    int lmin, lmax, p3;
    int spow;  // the forms of level l scale by 2^(l spow): 1 for 1/r, 2 for r/|r|^3
    long long loc_off[FMM_MAXDEPTH + 1];
    long long q_off[FMM_MAXDEPTH + 1];
    float *loc;
    const float *qlev;
    const float *kbar;  // [343][N], zero padded
    int *status;
    int inject_stall;   // test hook: the first stage's copies are withheld
};

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
    static constexpr int THREADS = 32 * (EPI + 2);      // + producer + MMA issuer
    static constexpr int KE = MODE == TC_BF16X3 ? 64 : 32;  // K elements per 128-byte chunk
    static constexpr int KC = (N + KE - 1) / KE;        // 128-byte K chunks
    static constexpr bool LO = MODE != TC_TF32X1;       // lo parts loaded and used
    static constexpr int BBYTES = N * 128;
    static constexpr int STAGE = 2 * TC_ABYTES + 2 * BBYTES;
    // ring depth: three 64 KB stages for N = 128 (one CTA per SM, 193 KB);
    // two otherwise (N = 64: two CTAs per SM of 2 x 48 KB; N = 224: 2 x 88 KB)
    static constexpr int STAGES = N == 128 ? 3 : 2;
    static constexpr int SMEM = STAGES * STAGE + 1024 + 128;
    static constexpr int TCOLS = 2 * N <= 64 ? 64 : (2 * N <= 128 ? 128 : (2 * N <= 256 ? 256 : 512));
    static constexpr int MINB = N <= 64 ? 2 : 1;
    static constexpr int COLS = N / CH;                 // columns per epilogue thread
};

template <int N, int MODE>
__global__ void __launch_bounds__(TcShape<N, MODE>::THREADS, TcShape<N, MODE>::MINB)
    k_m2l_tc(const __grid_constant__ TcParams prm) {
    typedef TcShape<N, MODE> Sh;
    extern __shared__ unsigned char smraw[];
    const uint32_t raw = tc::smem_u32(smraw);
    const uint32_t sbase = (raw + 1023u) & ~1023u;
    // barriers: full / empty per stage, rfull / rfree per TMEM region (two),
    // done, then the TMEM address slot (16 * STAGES + 40 <= 128 bytes)
    const uint32_t bars = sbase + Sh::STAGES * Sh::STAGE;
    const uint32_t full0 = bars, empty0 = bars + 8 * Sh::STAGES, rfull0 = bars + 16 * Sh::STAGES;
    const uint32_t rfree0 = rfull0 + 16;
    const uint32_t done = rfree0 + 16;  // every MMA of this CTA has completed
    const uint32_t tslot = done + 8;
    volatile uint32_t *tslot_ptr = reinterpret_cast<volatile uint32_t *>(smraw + (tslot - raw));

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // block -> level, target parity, tile of 8x4x4 coarse cells
    int l = prm.lmin;
    while (l < prm.lmax && (int)blockIdx.x >= prm.first_block[l + 1]) l++;
    const int rel = blockIdx.x - prm.first_block[l];
    const int H = 1 << (l - 1), P = H + 2;
    // levels with fewer than 8 x 4 x 4 coarse cells per parity take one tile,
    // partly outside the grid (those rows read the TMA fill and are not stored)
    const int ntx = (H + 7) / 8, nty = (H + 3) / 4, ntz = (H + 3) / 4;
    const int ntiles = ntx * nty * ntz;
    const int par = rel / ntiles, tile = rel % ntiles;
    const int X0 = (tile % ntx) * 8, Y0 = ((tile / ntx) % nty) * 4, Z0 = (tile / (ntx * nty)) * 4;
    const int bx = par & 1, by = (par >> 1) & 1, bz = par >> 2;

    if (threadIdx.x == 0) {
        for (int s = 0; s < Sh::STAGES; s++) {
            tc::mbar_init(full0 + 8 * s, 1);
            tc::mbar_init(empty0 + 8 * s, 1);
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

    if (warp == Sh::EPI && lane == 0) {
        // ---- TMA producer: (offset, K chunk) stages ----
        bool failed = false;
        int last_phase[TC_STAGES_MAX];
        for (int s = 0; s < TC_STAGES_MAX; s++) last_phase[s] = -1;
        int ox = -2 - bx - 1, oy = -2 - by, oz = -2 - bz, it = 0;
        while (!failed && next_offset(bx, by, bz, ox, oy, oz)) {
            const Off f = make_off(bx, by, bz, ox, oy, oz);
            const int cX = X0 + 1 + f.dX, cY = Y0 + 1 + f.dY, cZ = Z0 + 1 + f.dZ;
            for (int kc = 0; kc < Sh::KC; kc++, it++) {
                const int s = it % Sh::STAGES;
                const uint32_t ph = (uint32_t)(it / Sh::STAGES) & 1u;
                if (!tc::mbar_wait(empty0 + 8 * s, ph ^ 1u, TC_WAIT_CYCLES)) {
                    tc_wait_failed(prm.status, 1, l, it);
                    failed = true;
                    break;
                }
                const uint32_t st = sbase + s * Sh::STAGE;
                const uint32_t fb = full0 + 8 * s;
                const int kx = kc * Sh::KE;
                tc::mbar_expect_tx(fb, Sh::LO ? Sh::STAGE : TC_ABYTES + Sh::BBYTES);
                if (prm.inject_stall && it == 0) continue;  // armed, never filled (test hook)
                tc::tma_load_5d(st, &prm.phi_hi[l], fb, kx, cX, cY, cZ, f.spar);
                tc::tma_load_3d(st + 2 * TC_ABYTES, &prm.k_hi, fb, kx, 0, f.oi);
                if (Sh::LO) {
                    tc::tma_load_5d(st + TC_ABYTES, &prm.phi_lo[l], fb, kx, cX, cY, cZ, f.spar);
                    tc::tma_load_3d(st + 2 * TC_ABYTES + Sh::BBYTES, &prm.k_lo, fb, kx, 0, f.oi);
                }
                last_phase[s] = (int)ph;
            }
        }
        if (failed) {
            atomicOr(prm.status, ST_TIMEOUT);
            // let the copies already issued land before the CTA can exit
            for (int s = 0; s < Sh::STAGES; s++)
                if (last_phase[s] >= 0) tc::mbar_wait(full0 + 8 * s, (uint32_t)last_phase[s], TC_WAIT_CYCLES);
        }
    } else if (warp == Sh::EPI + 1 && lane == 0) {
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
                const int s = it % Sh::STAGES;
                const uint32_t ph = (uint32_t)(it / Sh::STAGES) & 1u;
                if (!tc::mbar_wait(full0 + 8 * s, ph, TC_WAIT_CYCLES)) {
                    tc_wait_failed(prm.status, 3, l, it);
                    failed = true;
                    break;
                }
                tc::fence_after_sync();
                const uint32_t st = sbase + s * Sh::STAGE;
#pragma unroll
                for (int k = 0; k < 4; k++) {  // 32 bytes of K per MMA (8 tf32 or 16 bf16)
                    const uint64_t ah = tc::desc_sw128(st + 32 * k);
                    const uint64_t al = tc::desc_sw128(st + TC_ABYTES + 32 * k);
                    const uint64_t bh = tc::desc_sw128(st + 2 * TC_ABYTES + 32 * k);
                    const uint64_t bl = tc::desc_sw128(st + 2 * TC_ABYTES + Sh::BBYTES + 32 * k);
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
                tc::mma_commit(empty0 + 8 * s);
            }
            if (!failed) tc::mma_commit(rfull0 + 8 * r);
        }
        if (failed) atomicOr(prm.status, ST_TIMEOUT);
        tc::mma_commit(done);  // always: the deallocation waits on it
    } else if (warp < Sh::EPI) {
        // ---- epilogue: TMEM lane = target cell; columns [c0, c0 + COLS) ----
        const int sub = warp & 3, cgrp = warp >> 2;
        const int c0 = cgrp * Sh::COLS;
        const int row = sub * 32 + lane;
        const int tx = row & 7, ty = (row >> 3) & 3, tz = row >> 5;
        const bool valid = X0 + tx < H && Y0 + ty < H && Z0 + tz < H;
        const float *q = prm.qlev + prm.q_off[l];
        float tot[Sh::COLS];
#pragma unroll
        for (int j = 0; j < Sh::COLS; j++) tot[j] = 0.0f;
        bool ok = true;
        int ox = -2 - bx - 1, oy = -2 - by, oz = -2 - bz;
        for (int i = 0; i < TC_NOFF; i++) {
            next_offset(bx, by, bz, ox, oy, oz);
            const Off f = make_off(bx, by, bz, ox, oy, oz);
            const float Qs = valid ? q[(((int64_t)f.spar * P + Z0 + tz + 1 + f.dZ) * P + Y0 + ty + 1 + f.dY) * P +
                                       X0 + tx + 1 + f.dX]
                                   : 0.0f;
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
        const int cx = 2 * (X0 + tx) + bx, cy = 2 * (Y0 + ty) + by, cz = 2 * (Z0 + tz) + bz;
        const int p3 = prm.p3;
        float *out = prm.loc + prm.loc_off[l] + (valid ? loc_cell(l, cx, cy, cz) : 0) * p3 + c0;
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

// Levels lmin..lmax of the grid charges, remapped from the padded layout (P =
// H + 2 per axis) into the operand layout (tc_level_extent per axis, zeros
// outside) and split into hi / lo parts.  One element = one (cell, b) of the
// operand layout.
struct SplitLevels {
    int lmin, lmax;
    long long src[FMM_MAXDEPTH + 2];  // first value of level l in the padded layout
    long long dst[FMM_MAXDEPTH + 2];  // first cell of level l in the operand layout
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
__global__ void k_split_tf32(const float *__restrict__ phi, SplitLevels L, float *__restrict__ hi,
                             float *__restrict__ lo, int p3, int p3s, int nearest) {
    const int q4 = p3s / 4;
    const int64_t c0 = L.dst[L.lmin], n = (L.dst[L.lmax + 1] - c0) * q4;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = c0 + i / q4;
        const int b0 = (int)(i % q4) * 4;
        int l;
        int64_t sc;
        const bool in = split_source(L, c, l, sc);
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

// BF16: hi = bf16(x), lo = bf16(x - hi), both rounded to nearest even; cell
// vectors of p3k values (zero padded, p3k % 64 == 0).  One thread per 4 values.
__global__ void k_split_bf16(const float *__restrict__ phi, SplitLevels L, __nv_bfloat16 *__restrict__ hi,
                             __nv_bfloat16 *__restrict__ lo, int p3, int p3k) {
    const int q4 = p3k / 4;
    const int64_t c0 = L.dst[L.lmin], n = (L.dst[L.lmax + 1] - c0) * q4;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = c0 + i / q4;
        const int b0 = (int)(i % q4) * 4;
        int l;
        int64_t sc;
        const bool in = split_source(L, c, l, sc);
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
static int launch_tc_kernel(const TcParams &prm, int blocks, cudaStream_t st) {
    typedef TcShape<N, MODE> Sh;
    static bool attr = false;
    if (!attr) {
        if (cudaFuncSetAttribute(k_m2l_tc<N, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 Sh::SMEM) != cudaSuccess)
            return FMM_ERR_CUDA;
        attr = true;
    }
    k_m2l_tc<N, MODE><<<blocks, Sh::THREADS, Sh::SMEM, st>>>(prm);
    return FMM_OK;
}

template <int MODE>
static int launch_tc_mode(int p3s, const TcParams &prm, int blocks, cudaStream_t st) {
    switch (p3s) {
    case 32: return launch_tc_kernel<32, MODE>(prm, blocks, st);
    case 64: return launch_tc_kernel<64, MODE>(prm, blocks, st);
    case 128: return launch_tc_kernel<128, MODE>(prm, blocks, st);
    case 224: return launch_tc_kernel<224, MODE>(prm, blocks, st);
    default: return FMM_ERR_UNSUPPORTED;
    }
}

int launch_m2l_tc(const Geom &g, const Ptrs<float> &P, const WsLayout &W, const void *k_hi_map,
                  const void *k_lo_map, const float *kbar, int lmin, int mode, int inject,
                  float *loc, int spow, bool split, cudaStream_t st, Tracer &tr) {
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
    tr.begin(FMM_STAGE_M2L, st);
    __nv_bfloat16 *hi16 = reinterpret_cast<__nv_bfloat16 *>(P.phihi);
    __nv_bfloat16 *lo16 = reinterpret_cast<__nv_bfloat16 *>(P.philo);
    if (split) {
        if (bf16)
            k_split_bf16<<<152 * 8, 256, 0, st>>>(P.phi, SL, hi16, lo16, p3, pk);
        else
            k_split_tf32<<<152 * 8, 256, 0, st>>>(P.phi, SL, P.phihi, P.philo, p3, p3s, mode == FMM_TC_TF32X1);
        tr.count();
    }
    TcParams prm;
    memset(&prm, 0, sizeof(prm));
    int blocks = 0;
    for (int l = lmin; l <= depth; l++) {
        const int64_t cl = tc_level_first(l);  // first cell of level l (operand layout)
        const void *bh = bf16 ? (const void *)(hi16 + cl * pk) : (const void *)(P.phihi + cl * p3s);
        const void *bl = bf16 ? (const void *)(lo16 + cl * pk) : (const void *)(P.philo + cl * p3s);
        int rc = encode_phi_map(&prm.phi_hi[l], bh, l, pk, bf16);
        if (!rc) rc = encode_phi_map(&prm.phi_lo[l], bl, l, pk, bf16);
        if (rc) return rc;
        prm.first_block[l] = blocks;
        const int H = 1 << (l - 1);
        blocks += 8 * ((H + 7) / 8) * ((H + 3) / 4) * ((H + 3) / 4);
        prm.loc_off[l] = W.loc_level[l];
        prm.q_off[l] = W.q_level[l];
    }
    prm.first_block[depth + 1] = blocks;
    memcpy(&prm.k_hi, k_hi_map, sizeof(CUtensorMap));
    memcpy(&prm.k_lo, k_lo_map, sizeof(CUtensorMap));
    prm.lmin = lmin;
    prm.lmax = depth;
    prm.p3 = p3;
    prm.spow = spow;
    prm.loc = loc;
    prm.qlev = P.qlev;
    prm.kbar = kbar;
    prm.status = &P.hdr->status;
    prm.inject_stall = inject == FMM_INJECT_TC_STALL;
    int rc = mode == FMM_TC_BF16X3   ? launch_tc_mode<TC_BF16X3>(p3s, prm, blocks, st)
             : mode == FMM_TC_TF32X1 ? launch_tc_mode<TC_TF32X1>(p3s, prm, blocks, st)
                                     : launch_tc_mode<TC_TF32X3>(p3s, prm, blocks, st);
    tr.count();
    tr.end();
    return rc;
}

}  // namespace fmm

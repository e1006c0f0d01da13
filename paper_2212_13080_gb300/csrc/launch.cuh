// Kernel launches that a batched evaluation can merge across systems.
//
// A batchable kernel is a functor K: its parameters are members, its body is
// `__device__ void run(int block, int nblocks) const` (the block index and
// the grid size it would have in a launch of its own), and K::BS / K::MINB
// are its block size and the blocks per SM its register budget must allow.
// A single-system evaluation launches the kernel's named wrapper with K as
// its one parameter.  A batched evaluation records every launch of every
// system (Tracer::rec) instead, then launches each call site once for all
// systems (kb_many<K>): block b of the merged grid runs block b - first[s] of
// system s, first[] being the prefix of the systems' block counts, with
// system s's K read from a device array.  The body is the same code in both
// forms, so a system's results are the same bit for bit.
#pragma once
#include <cstring>
#include <vector>

#include "fmm_internal.cuh"

namespace fmm {

// merged form: every system's blocks in one grid (K::BS = 0: a kernel
// without launch bounds)
template <class K>
__device__ __forceinline__ void kb_run(const K *__restrict__ ks, const int *__restrict__ first, int nsys) {
    const int b = blockIdx.x;
    int lo = 0, hi = nsys - 1;  // the last system whose first block is <= b (it has blocks)
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(first + mid) <= b) lo = mid;
        else hi = mid - 1;
    }
    const int f0 = __ldg(first + lo);
    ks[lo].run(b - f0, __ldg(first + lo + 1) - f0);
}
// launch bounds as the functor's named kernel has them: block size and
// minimum blocks per SM (MINB > 0), the block size only (MINB = 0), none (BS = 0)
template <class K>
__global__ void __launch_bounds__(K::BS, K::MINB) kb_many(const K *__restrict__ ks, const int *__restrict__ first,
                                                          int nsys) {
    kb_run(ks, first, nsys);
}
template <class K>
__global__ void __launch_bounds__(K::BS) kb_many_bs(const K *__restrict__ ks, const int *__restrict__ first, int nsys) {
    kb_run(ks, first, nsys);
}
template <class K>
__global__ void kb_many_nolb(const K *__restrict__ ks, const int *__restrict__ first, int nsys) {
    kb_run(ks, first, nsys);
}

template <class K>
void kb_launch_many(const void *ks, const int *first, int nsys, int total, int threads, size_t smem,
                    cudaStream_t st) {
    const K *k = reinterpret_cast<const K *>(ks);
    if constexpr (K::BS > 0 && K::MINB > 0)
        kb_many<K><<<total, threads, smem, st>>>(k, first, nsys);
    else if constexpr (K::BS > 0)
        kb_many_bs<K><<<total, threads, smem, st>>>(k, first, nsys);
    else
        kb_many_nolb<K><<<total, threads, smem, st>>>(k, first, nsys);
}
template <class K>
void kb_set_smem(size_t smem) {
    if constexpr (K::BS > 0 && K::MINB > 0)
        cudaFuncSetAttribute(kb_many<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    else if constexpr (K::BS > 0)
        cudaFuncSetAttribute(kb_many_bs<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    else
        cudaFuncSetAttribute(kb_many_nolb<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

// A launch of one system, recorded for merging: call sites (tag: site and
// level or component) of different systems with equal tags merge.
struct LaunchRec {
    int tag;
    int near;  // issued on the near-field stream (it joins the rest at a marker)
    int blocks, threads;
    size_t smem;
    size_t ksize, kalign;
    std::vector<unsigned char> k;
    void (*many)(const void *, const int *, int, int, int, size_t, cudaStream_t);
    void (*set_smem)(size_t);
};

// Call-site tags: a site number per launch site, and a sub-index (level,
// kernel component) where one site launches several times per evaluation.
#define FMM_TAG(site, sub) (((site) << 8) | (sub))
enum LaunchSite {
    S_ZERO_HDR = 1, S_ZERO_LEAF, S_SPLIT_COUNT, S_SCAN_BLOCKS_E, S_SCAN_APPLY_E, S_EMIT,
    S_SCAN_ONE, S_SCAN_REDUCE, S_SCAN_BLOCKS, S_SCAN_APPLY, S_SCATTER, S_LEAF_GATHER,
    S_ZERO_PORD, S_NF_COUNT, S_NF_FILL, S_P2P,
    S_P2M, S_HALO, S_M2M, S_LATTICE, S_M2L_SIMT, S_M2L_REDUCE,
    S_SPLIT_TC, S_OCC_COUNT, S_OCC_OFFSETS, S_OCC_SCATTER, S_M2L_TC,
    S_L2L, S_ZERO_SLIST, S_SPLIT_LIST, S_SPLIT_DELTA, S_L2P,
    S_ZERO_ENERGY, S_UNSPLIT, S_ENERGY_FINAL, S_MARK_VALID, S_JOIN_NEAR, S_M2L_TCX
};

template <class K>
inline void launch_k(Tracer &tr, int tag, void (*named)(K), const K &k, int blocks, int threads, size_t smem,
                     cudaStream_t st) {
    if (tr.rec) {
        LaunchRec r;
        r.tag = tag;
        r.near = tr.near && st == tr.near;
        r.blocks = blocks;
        r.threads = threads;
        r.smem = smem;
        r.ksize = sizeof(K);
        r.kalign = alignof(K);
        r.k.resize(sizeof(K));
        memcpy(r.k.data(), &k, sizeof(K));
        r.many = kb_launch_many<K>;
        r.set_smem = kb_set_smem<K>;
        tr.rec->push_back(std::move(r));
        return;
    }
    if (blocks > 0) named<<<blocks, threads, smem, st>>>(k);
}

// a point of the recorded sequence where the work recorded on the near-field
// stream must be complete (many = nullptr: launches nothing)
inline void record_marker(Tracer &tr, int tag) {
    LaunchRec r;
    r.tag = tag;
    r.near = 0;
    r.blocks = r.threads = 0;
    r.smem = r.ksize = r.kalign = 0;
    r.many = nullptr;
    r.set_smem = nullptr;
    tr.rec->push_back(std::move(r));
}

// Zeroing of device memory (a memset that a batched evaluation can merge):
// words [0, nw) of p, four per thread.
struct KZero {
    static constexpr int BS = 256, MINB = 1;  // launched with BS threads
    int *p;
    int64_t nw;
    __device__ void run(int bid, int nblk) const {
        for (int64_t i = (int64_t)bid * BS + threadIdx.x; 4 * i < nw; i += (int64_t)nblk * BS) {
            const int64_t w = 4 * i;
            if (w + 4 <= nw && ((reinterpret_cast<uintptr_t>(p + w) & 15) == 0)) {
                *reinterpret_cast<int4 *>(p + w) = make_int4(0, 0, 0, 0);
            } else {
                for (int64_t j = w; j < nw && j < w + 4; j++) p[j] = 0;
            }
        }
    }
};
void zero_words(Tracer &tr, int tag, void *p, size_t bytes, cudaStream_t st);

}  // namespace fmm

// ops_impl.cuh -- kernel launchers for one element type; each ops_<type>.cu
// instantiates them once so the element types compile in parallel.
#pragma once

#include "base.cuh"
#include "classify.cuh"
#include "graph.cuh"
#include "level.cuh"
#include "sorter.h"

namespace ipsgpu {

template <class T>
struct OpsImpl {
    typedef typename T::K K;
    static size_t classify_smem(const Sorter *s) { return ClsSmem<T>::bytes(s->k, s->b); }
    static size_t classify_smem_bytes(uint32_t k, uint32_t b) { return ClsSmem<T>::bytes(k, b); }
    static size_t sample_smem() {
        return (max_sort_sample<K>() + kMaxClasses) * sizeof(K) +
               sizeof(uint32_t) * (2 * kMaxClasses + 34);
    }

    // Raises the dynamic shared-memory limit of a kernel to the most the
    // device allows next to its static shared memory.  The attribute
    // belongs to the kernel (process-wide), so it is never set to what one
    // sorter needs: a later sorter with smaller blocks would lower it under
    // every earlier one.  Each launch still asks for its own size.
    template <class F>
    static cudaError_t raise_smem_limit(F *kernel, int optin) {
        cudaFuncAttributes fa;
        cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
        if (e != cudaSuccess) return e;
        return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    optin - (int)fa.sharedSizeBytes);
    }
    // Kernel attributes; for a sorter (nsm and b set) also the number of
    // permutation CTAs that are resident at once, which sizes the level's
    // virtual CTAs.
    static cudaError_t init(Sorter *s) {
        int dev = 0, optin = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess)
            e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e == cudaSuccess) e = raise_smem_limit(k_classify<T>, optin);
        if (e == cudaSuccess) e = raise_smem_limit(k_sample_tree<T>, optin);
        if (e == cudaSuccess) e = raise_smem_limit(k_base<T, BaseLarge>, optin);
        if (e == cudaSuccess) e = raise_smem_limit(k_base<T, BaseSmall>, optin);
        if (e == cudaSuccess && s && s->nsm > 0 && s->b > 0) {
            int occ = 0;
            const int nv = block_units(s->b * T::D);
            if (nv == 1)
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_permute<T, 1>, kPermuteThreads, 0);
            else if (nv == 2)
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_permute<T, 2>, kPermuteThreads, 0);
            else
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_permute<T, 4>, kPermuteThreads, 0);
            s->perm_ctas = (uint32_t)s->nsm * (uint32_t)(occ > 0 ? occ : 1);
        }
        return e;
    }

    template <int NV>
    static void launch_moves(Sorter *s, const LevelArgs &a, const LevelGrids &g, cudaStream_t st,
                             double lvl) {
        s->tbegin(KK_FIXUP, 0, st);
        k_fixup<T, NV><<<s->nsm * 4, kAuxThreads, 0, st>>>(a);
        s->tend(st);
        s->tbegin(KK_PERMUTE, 2 * lvl, st);
        k_permute<T, NV><<<g.cta, kPermuteThreads, 0, st>>>(a);
        s->tend(st);
    }

    // One partitioning level.  g holds the grid of each kernel: the exact
    // work counts for a host-planned batch, or fixed persistent grids when
    // the counts live in device memory (a.cnt != nullptr).
    static cudaError_t level(Sorter *s, const LevelArgs &a, const LevelGrids &g, cudaStream_t st) {
        const double lvl = (double)s->level_elems * T::D;
        cudaError_t e;
        // a device-planned wave clears the move counter in k_g_plan
        if (!a.cnt && (e = cudaMemsetAsync(a.nmoves, 0, sizeof(uint32_t), st)) != cudaSuccess)
            return e;
        s->tbegin(KK_SAMPLE, 0, st);
        k_sample_tree<T><<<g.seg, kSampleThreads, sample_smem(), st>>>(a);
        s->tend(st);
        s->tbegin(KK_CLASSIFY, 2 * lvl, st);
        k_classify<T><<<g.stripe, ClsCfg<T>::NT, classify_smem(s), st>>>(a);
        s->tend(st);
        // a classification that did not launch left no counts: stop before
        // the kernels that would read the previous level's
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        s->tbegin(KK_PREP, 0, st);
        k_prep<<<g.seg, kAuxThreads, 0, st>>>(a);
        s->tend(st);
        switch (block_units(s->b * T::D)) {
        case 1: launch_moves<1>(s, a, g, st, lvl); break;
        case 2: launch_moves<2>(s, a, g, st, lvl); break;
        default: launch_moves<4>(s, a, g, st, lvl); break;
        }
        s->tbegin(KK_STAGE, 0, st);
        k_stage<T><<<g.seg, kAuxThreads, 0, st>>>(a);
        s->tend(st);
        s->tbegin(KK_FILL, 0, st);
        k_fill<T><<<g.cls, kAuxThreads, 0, st>>>(a);
        s->tend(st);
        return cudaGetLastError();
    }

    static cudaError_t base(Sorter *s, const uint64_t *d_segs, uint32_t nsegs,
                            const uint32_t *nsegs_dev, uint32_t grid, cudaStream_t st) {
        if (grid == 0) return cudaSuccess;
        // segments that fit the small shape: two CTAs per SM; the rest: one
        const uint64_t small_cap = (uint64_t)BaseSmall::BUF / T::D;
        s->tbegin(KK_BASE, 2.0 * (double)s->level_elems * T::D, st);
        k_base<T, BaseSmall><<<2 * grid, BaseSmall::NT, base_smem_bytes<BaseSmall>(), st>>>(
            d_segs, nsegs, nsegs_dev, s->d_status, 0ull, small_cap);
        k_base<T, BaseLarge><<<grid, BaseLarge::NT, base_smem_bytes<BaseLarge>(), st>>>(
            d_segs, nsegs, nsegs_dev, s->d_status, small_cap, ~0ull);
        s->tend(st);
        return cudaGetLastError();
    }

    static cudaError_t detect(Sorter *s, const unsigned char *data, uint64_t n,
                              unsigned long long *mm, cudaStream_t st) {
        uint64_t chunks = (n + kDetectChunk - 1) / kDetectChunk;
        uint32_t grid = (uint32_t)(chunks < (uint64_t)s->nsm * 8 ? chunks : (uint64_t)s->nsm * 8);
        if (grid == 0) grid = 1;
        // with mm (radix) the pass reads every element; without it, it stops
        // once both properties are refuted, after an amount read that only
        // the device knows, so no bytes are attributed to the launch
        s->tbegin(KK_DETECT, mm ? (double)n * T::D : 0.0, st);
        k_detect<T><<<grid, kDetectThreads, 0, st>>>(data, n, s->d_flags, mm);
        s->tend(st);
        return cudaGetLastError();
    }

    static cudaError_t reverse(Sorter *s, unsigned char *data, uint64_t n, cudaStream_t st) {
        uint64_t pairs = n / 2;
        uint64_t g = (pairs + 255) / 256;
        uint32_t grid = (uint32_t)(g < (uint64_t)s->nsm * 16 ? g : (uint64_t)s->nsm * 16);
        if (grid == 0) return cudaSuccess;
        // moves 2 n D bytes only when the input was non-increasing (decided on
        // the device), so no bytes are attributed to the launch
        s->tbegin(KK_REVERSE, 0, st);
        k_reverse<T><<<grid, 256, 0, st>>>(data, n, s->d_flags);
        s->tend(st);
        return cudaGetLastError();
    }

    static cudaError_t classify_ids(Sorter *s, const LevelArgs &a, uint32_t *out, cudaStream_t st) {
        s->tbegin(KK_SAMPLE, 0, st);
        k_sample_tree<T><<<1, kSampleThreads, sample_smem(), st>>>(a);
        s->tend(st);
        uint64_t n = s->level_elems;
        uint64_t g = (n + kAuxThreads - 1) / kAuxThreads;
        uint32_t grid = (uint32_t)(g < (uint64_t)s->nsm * 16 ? g : (uint64_t)s->nsm * 16);
        if (grid == 0) grid = 1;
        s->tbegin(KK_CLASSIFY_IDS, (double)n * (T::D + 4), st);
        k_classify_ids<T><<<grid, kAuxThreads, 0, st>>>(a, out);
        s->tend(st);
        return cudaGetLastError();
    }

    // One wave of the device-planned recursion (graph.cuh).  Every launch
    // has a fixed grid and reads its work counts from device memory, so the
    // same sequence serves as the body of the graph's WHILE loop (in_graph)
    // and as one step of the host-driven loop used when timing kernels.
    static cudaError_t wave(Sorter *s, const GraphArgs &ga, cudaStream_t st, int in_graph,
                            cudaGraphConditionalHandle h) {
        const uint32_t big = (uint32_t)s->nsm * 8;
        s->tbegin(KK_PLAN, 0, st);
        k_g_feed<<<big, kAuxThreads, 0, st>>>(ga);
        k_g_plan<T><<<1, kPlanThreads, 0, st>>>(ga);
        k_g_fill_stripes<T><<<big, kAuxThreads, 0, st>>>(ga);
        s->tend(st);
        LevelArgs a = ga.lv;
        a.cnt = &ga.state->counts;
        a.stripe_first = ga.stripe_first;
        LevelGrids g;
        g.seg = (uint32_t)s->nsm * 4;
        g.stripe = ga.nparts;  // one classification part per CTA
        g.cta = s->perm_ctas;
        g.cls = big;
        cudaError_t e;
        if ((e = level(s, a, g, st)) != cudaSuccess) return e;
        s->tbegin(KK_PLAN, 0, st);
        k_g_emit<T><<<big, kAuxThreads, 0, st>>>(ga);
        s->tend(st);
        if ((e = base(s, ga.base_list, 0, &ga.state->base_count, s->nsm, st)) != cudaSuccess)
            return e;
        k_g_advance<<<1, 32, 0, st>>>(ga, h, in_graph);
        return cudaGetLastError();
    }

    static TypeOps make() {
        TypeOps o;
        o.D = T::D;
        o.key_bytes = sizeof(K);
        o.init = &init;
        o.classify_smem_bytes = &classify_smem_bytes;
        o.level = &level;
        o.base = &base;
        o.detect = &detect;
        o.reverse = &reverse;
        o.classify_ids = &classify_ids;
        o.wave = &wave;
        return o;
    }
};

}  // namespace ipsgpu

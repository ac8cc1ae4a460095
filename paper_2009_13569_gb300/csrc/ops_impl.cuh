// ops_impl.cuh -- kernel launchers for one element type; each ops_<type>.cu
// instantiates them once so the element types compile in parallel.
#pragma once

#include "base.cuh"
#include "classify.cuh"
#include "level.cuh"
#include "sorter.h"

namespace ipsgpu {

template <class T>
struct OpsImpl {
    typedef typename T::K K;
    static size_t classify_smem(const Sorter *s) { return ClsSmem<T>::bytes(s->b); }
    static size_t sample_smem() {
        return (kMaxSortSample + kMaxClasses) * sizeof(K) + sizeof(uint32_t) * (2 * kMaxClasses + 34);
    }

    static cudaError_t init(Sorter *s) {
        cudaError_t e;
        e = cudaFuncSetAttribute(k_classify<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)classify_smem(s));
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(k_sample_tree<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sample_smem());
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(k_base<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)base_smem_bytes());
        return e;
    }

    static cudaError_t level(Sorter *s, uint32_t nseg, uint32_t nstripe, uint32_t ncta,
                             const unsigned char *given_spl, cudaStream_t st) {
        LevelArgs a = s->args(nseg, nstripe, given_spl);
        const double lvl = (double)s->level_elems * T::D;
        cudaError_t e;
        if ((e = cudaMemsetAsync(s->d_nmoves, 0, sizeof(uint32_t), st)) != cudaSuccess) return e;
        s->tbegin(KK_SAMPLE, 0, st);
        k_sample_tree<T><<<nseg, kSampleThreads, sample_smem(), st>>>(a);
        s->tend(st);
        s->tbegin(KK_CLASSIFY, 2 * lvl, st);
        k_classify<T><<<nstripe, ClsCfg<T>::NT, classify_smem(s), st>>>(a);
        s->tend(st);
        s->tbegin(KK_PREP, 0, st);
        k_prep<<<nseg, kAuxThreads, 0, st>>>(a);
        s->tend(st);
        s->tbegin(KK_FIXUP, 0, st);
        k_fixup<T><<<s->nsm * 4, kAuxThreads, 0, st>>>(a);
        s->tend(st);
        s->tbegin(KK_PERMUTE, 2 * lvl, st);
        k_permute<T><<<ncta, kPermuteThreads, 0, st>>>(a, s->d_cta_seg);
        s->tend(st);
        s->tbegin(KK_STAGE, 0, st);
        k_stage<T><<<nseg, kAuxThreads, 0, st>>>(a);
        s->tend(st);
        s->tbegin(KK_FILL, 0, st);
        k_fill<T><<<dim3(kMaxClasses, nseg), kAuxThreads, 0, st>>>(a);
        s->tend(st);
        return cudaGetLastError();
    }

    static cudaError_t pack(Sorter *s, uint32_t nseg, cudaStream_t st) {
        LevelArgs a = s->args(nseg, 0, nullptr);
        s->tbegin(KK_PACK, 0, st);
        k_pack_results<<<nseg, kAuxThreads, 0, st>>>(a, s->d_res);
        s->tend(st);
        return cudaGetLastError();
    }

    static cudaError_t base(Sorter *s, unsigned char *data, const uint64_t *d_segs, uint32_t nsegs,
                            cudaStream_t st) {
        if (nsegs == 0) return cudaSuccess;
        uint32_t grid = nsegs < (uint32_t)s->nsm * 64 ? nsegs : (uint32_t)s->nsm * 64;
        s->tbegin(KK_BASE, 2.0 * (double)s->level_elems * T::D, st);
        k_base<T><<<grid, kBaseThreads, base_smem_bytes(), st>>>(data, d_segs, nsegs, s->d_status);
        s->tend(st);
        return cudaGetLastError();
    }

    static cudaError_t detect(Sorter *s, const unsigned char *data, uint64_t n, cudaStream_t st) {
        uint64_t chunks = (n + kDetectChunk - 1) / kDetectChunk;
        uint32_t grid = (uint32_t)(chunks < (uint64_t)s->nsm * 8 ? chunks : (uint64_t)s->nsm * 8);
        if (grid == 0) grid = 1;
        s->tbegin(KK_DETECT, 0, st);
        k_detect<T><<<grid, kDetectThreads, 0, st>>>(data, n, s->d_flags);
        s->tend(st);
        return cudaGetLastError();
    }

    static cudaError_t reverse(Sorter *s, unsigned char *data, uint64_t n, cudaStream_t st) {
        uint64_t pairs = n / 2;
        uint64_t g = (pairs + 255) / 256;
        uint32_t grid = (uint32_t)(g < (uint64_t)s->nsm * 16 ? g : (uint64_t)s->nsm * 16);
        if (grid == 0) return cudaSuccess;
        s->tbegin(KK_REVERSE, 2.0 * n * T::D, st);
        k_reverse<T><<<grid, 256, 0, st>>>(data, n);
        s->tend(st);
        return cudaGetLastError();
    }

    static cudaError_t classify_ids(Sorter *s, const unsigned char *given_spl, uint32_t *out,
                                    cudaStream_t st) {
        LevelArgs a = s->args(1, 0, given_spl);
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

    static TypeOps make() {
        TypeOps o;
        o.D = T::D;
        o.key_bytes = sizeof(K);
        o.init = &init;
        o.level = &level;
        o.pack = &pack;
        o.base = &base;
        o.detect = &detect;
        o.reverse = &reverse;
        o.classify_ids = &classify_ids;
        return o;
    }
};

}  // namespace ipsgpu

// base.cuh -- kernels around the partitioning levels:
//   k_detect   one pass that tells whether the input is non-decreasing or
//              non-increasing (Sec. 5: sorted inputs return at once,
//              decreasing ones are reversed); it stops as soon as both
//              properties are refuted
//   k_reverse  in-place reversal
//   k_base     the base case: every segment small enough for one SM's
//              shared memory is sorted there (the GPU replacement of the
//              insertion-sort base case of Sec. 5)
#pragma once

#include "common.cuh"

namespace ipsgpu {

constexpr int kDetectThreads = 256;
constexpr int kDetectChunk = 8192;
constexpr int kBaseThreads = 512;
constexpr int kBaseDigitBits = 11;       // at most 2048 sub-buckets per pass
constexpr int kBaseInsertion = 24;       // sub-buckets up to this size: insertion sort
constexpr int kBaseStack = 2048;         // pending ranges: >= 196608 B / 4 B / 25


// second-level radix key: non-zero only for keys wider than 64 bits
template <class T>
__device__ __forceinline__ uint64_t rk_lo(const typename T::E &e) { return 0; }
template <>
__device__ __forceinline__ uint64_t rk_lo<TRec100>(const TRec100::E &e) {
    return TRec100::key(e).lo;
}

template <class T>
__global__ void __launch_bounds__(kDetectThreads) k_detect(const unsigned char *data, uint64_t n,
                                                           int *flags) {
    typedef typename T::E E;
    const E *a = reinterpret_cast<const E *>(data);
    volatile int *vf = flags;
    for (uint64_t c0 = (uint64_t)blockIdx.x * kDetectChunk; c0 + 1 < n;
         c0 += (uint64_t)gridDim.x * kDetectChunk) {
        if (vf[0] == 0 && vf[1] == 0) return;
        bool inc = true, dec = true;
        const uint64_t c1 = min(c0 + kDetectChunk, n - 1);
        for (uint64_t i = c0 + threadIdx.x; i < c1; i += blockDim.x) {
            typename T::K k0 = T::key(a[i]), k1 = T::key(a[i + 1]);
            if (k1 < k0) inc = false;
            if (k0 < k1) dec = false;
        }
        if (!inc) flags[0] = 0;
        if (!dec) flags[1] = 0;
    }
}

template <class T>
__global__ void __launch_bounds__(256) k_reverse(unsigned char *data, uint64_t n) {
    typedef typename T::E E;
    E *a = reinterpret_cast<E *>(data);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n / 2;
         i += (uint64_t)gridDim.x * blockDim.x) {
        E x = a[i], y = a[n - 1 - i];
        a[i] = y;
        a[n - 1 - i] = x;
    }
}

template <class T>
__device__ __forceinline__ typename T::K shfl_key(typename T::K k, int src) {
    return __shfl_sync(0xffffffffu, k, src);
}
template <>
__device__ __forceinline__ Key80 shfl_key<TRec100>(Key80 k, int src) {
    Key80 r;
    r.hi = __shfl_sync(0xffffffffu, k.hi, src);
    r.lo = __shfl_sync(0xffffffffu, k.lo, src);
    return r;
}

// Sorts each listed segment (segs[2i] = begin, segs[2i+1] = n, n <= smax)
// in place.  Per segment: the elements are read from global memory, spread
// by an MSD radix digit of (key - min) into shared memory, and each
// sub-bucket is finished by insertion sort or, if larger, by another pass.
// A pass reads its range from global memory (the range's final position,
// which the previous pass left there) and scatters it into the same range
// of the shared buffer.
template <class T>
__global__ void __launch_bounds__(kBaseThreads, 1) k_base(unsigned char *data,
                                                          const uint64_t *segs, uint32_t nsegs,
                                                          int *status) {
    typedef typename T::E E;
    typedef typename T::K K;
    constexpr int ND = 1 << kBaseDigitBits;
    extern __shared__ __align__(16) unsigned char smem[];
    // layout: buf | stk (8-byte entries, kept 8-byte aligned) | off | cur | wtmp
    E *buf = reinterpret_cast<E *>(smem);
    uint2 *stk = reinterpret_cast<uint2 *>(smem + kBaseSmemBytes);        // kBaseStack
    uint32_t *off = reinterpret_cast<uint32_t *>(stk + kBaseStack);       // ND + 1
    uint32_t *cur = off + ND + 1;                                         // ND
    uint32_t *wtmp = cur + ND;                                            // 34
    __shared__ unsigned long long red[2][32];
    __shared__ uint32_t sp;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = kBaseThreads / 32;

    for (uint32_t si = blockIdx.x; si < nsegs; si += gridDim.x) {
        const uint64_t begin = segs[2 * si], n = segs[2 * si + 1];
        E *g = reinterpret_cast<E *>(data) + begin;
        if (n <= 1) continue;
        if (n <= 32) {
            // rank sort by one warp
            if (warp == 0) {
                E x;
                K k = T::max_key();
                if (lane < (int)n) {
                    x = g[lane];
                    k = T::key(x);
                }
                uint32_t rank = 0;
                for (int j = 0; j < (int)n; j++) {
                    K kj = shfl_key<T>(k, j);
                    if (kj < k || (!(k < kj) && j < lane)) rank++;
                }
                __syncwarp();
                if (lane < (int)n) g[rank] = x;
            }
            __syncthreads();
            continue;
        }
        if (tid == 0) {
            sp = 1;
            stk[0] = make_uint2(0, (uint32_t)n);
        }
        __syncthreads();
        while (sp > 0) {
            const uint2 top = stk[sp - 1];
            __syncthreads();
            if (tid == 0) sp--;
            const uint32_t a0 = top.x, len = top.y;
            // min / max of the radix key over the range (two key words)
            int mode = 0;  // 0: high word, 1: low word (keys wider than 64 bits)
            uint64_t mn = 0, rng = 0;
            for (int pass = 0; pass < 2; pass++) {
                unsigned long long lmin = ~0ull, lmax = 0;
                for (uint32_t i = tid; i < len; i += kBaseThreads) {
                    const E x = g[a0 + i];
                    uint64_t v = pass == 0 ? T::rkey(x) : rk_lo<T>(x);
                    lmin = min(lmin, (unsigned long long)v);
                    lmax = max(lmax, (unsigned long long)v);
                }
                for (int o = 16; o > 0; o >>= 1) {
                    lmin = min(lmin, __shfl_xor_sync(0xffffffffu, lmin, o));
                    lmax = max(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
                }
                if (lane == 0) {
                    red[0][warp] = lmin;
                    red[1][warp] = lmax;
                }
                __syncthreads();
                unsigned long long gmin = red[0][0], gmax = red[1][0];
                for (int w = 1; w < NW; w++) {
                    gmin = min(gmin, red[0][w]);
                    gmax = max(gmax, red[1][w]);
                }
                __syncthreads();
                mode = pass;
                mn = gmin;
                rng = gmax - gmin;
                if (rng != 0 || sizeof(typename T::K) <= 8) break;
            }
            if (rng == 0) continue;  // all keys equal: the range is final
            const uint32_t nbits = 64 - __clzll((long long)rng);
            uint32_t want = 1;
            while (want < kBaseDigitBits && ((uint64_t)6 << want) < len) want++;
            const uint32_t dbits = min(nbits, want);
            const uint32_t shift = nbits - dbits;
            const uint32_t nd = 1u << dbits;
            for (uint32_t d = tid; d < nd; d += kBaseThreads) cur[d] = 0;
            __syncthreads();
            for (uint32_t i = tid; i < len; i += kBaseThreads) {
                const E x = g[a0 + i];
                uint64_t v = mode == 0 ? T::rkey(x) : rk_lo<T>(x);
                atomicAdd(&cur[(uint32_t)((v - mn) >> shift)], 1u);
            }
            __syncthreads();
            cta_exclusive_scan<uint32_t>(cur, off, (int)nd, wtmp);
            if (tid == 0) off[nd] = len;
            for (uint32_t d = tid; d < nd; d += kBaseThreads) cur[d] = off[d];
            __syncthreads();
            for (uint32_t i = tid; i < len; i += kBaseThreads) {
                const E x = g[a0 + i];
                uint64_t v = mode == 0 ? T::rkey(x) : rk_lo<T>(x);
                uint32_t p = atomicAdd(&cur[(uint32_t)((v - mn) >> shift)], 1u);
                buf[a0 + p] = x;
            }
            __syncthreads();
            for (uint32_t d = tid; d < nd; d += kBaseThreads) {
                const uint32_t o = a0 + off[d], c = off[d + 1] - off[d];
                if (c <= 1) continue;
                if (c <= kBaseInsertion) {
                    for (uint32_t i = 1; i < c; i++) {
                        E x = buf[o + i];
                        K kx = T::key(x);
                        uint32_t j = i;
                        while (j > 0 && kx < T::key(buf[o + j - 1])) {
                            buf[o + j] = buf[o + j - 1];
                            j--;
                        }
                        buf[o + j] = x;
                    }
                } else {
                    uint32_t q = atomicAdd(&sp, 1u);
                    if (q < kBaseStack)
                        stk[q] = make_uint2(o, c);
                    else
                        set_status(status, IPSGPU_E_INTERNAL);
                }
            }
            __syncthreads();
            if (sp > kBaseStack) {
                if (tid == 0) sp = kBaseStack;
                __syncthreads();
            }
            for (uint32_t i = tid; i < len; i += kBaseThreads) g[a0 + i] = buf[a0 + i];
            __syncthreads();
        }
        __syncthreads();
    }
}

inline size_t base_smem_bytes() {
    return kBaseSmemBytes + sizeof(uint32_t) * ((1 << kBaseDigitBits) * 2 + 1) +
           sizeof(uint2) * kBaseStack + sizeof(uint32_t) * 34 + 16;
}

}  // namespace ipsgpu

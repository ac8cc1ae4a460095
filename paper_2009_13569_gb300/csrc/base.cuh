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

#include "classify.cuh"
#include "common.cuh"

namespace ipsgpu {

constexpr int kDetectThreads = 256;
constexpr int kDetectChunk = 8192;
constexpr int kBaseThreads = 1024;
constexpr int kBaseDigitBits = 14;       // at most 16384 sub-buckets per pass
constexpr int kBaseInsertion = 24;       // sub-buckets up to this size: ranked directly
constexpr int kBaseStack = 256;          // pending large ranges: >= 188416 B / 4 B / 513
constexpr int kBaseSmall = 512;          // ranges up to this size are finished by one warp
constexpr int kBaseSmallStack = 2048;    // pending small ranges: >= 188416 B / 4 B / 25
constexpr int kBasePeel = 4;             // distinct keys a small range is peeled by
constexpr uint32_t kBaseSpin = 1u << 22;  // polls of a bounded wait on a segment's bulk copy


// Radix-key word w < T::kKeyWords of an element, most significant first
// (word 0 is T::rkey): keys wider than 64 bits go on in later words.
template <class T>
__device__ __forceinline__ uint64_t rk_word(const typename T::E &e, int w) {
    return T::rkey(e);
}
template <>
__device__ __forceinline__ uint64_t rk_word<TRec100>(const TRec100::E &e, int w) {
    return w == 0 ? TRec100::rkey(e) : (uint64_t)TRec100::key(e).lo;
}
template <>
__device__ __forceinline__ uint64_t rk_word<TQuartet>(const TQuartet::E &e, int w) {
    return w == 0 ? e.a : (w == 1 ? e.b : e.c);
}

// One pass over the input (Sec. 5): flags[0] stays set iff it is
// non-decreasing, flags[1] iff it is non-increasing.  Each block reduces its
// chunk's verdict with barrier votes and clears a flag at most once (a store
// per thread to one word would serialise on it); a block stops as soon as
// both flags are clear (the decision is block-uniform).  With mm set (radix
// sorts) the pass reads everything and also leaves the minimum and maximum
// radix key in mm[0], mm[1] (preset to ~0 and 0), from which the first digit
// is placed at the highest bit where they differ.
template <class T>
__global__ void __launch_bounds__(kDetectThreads) k_detect(const unsigned char *data, uint64_t n,
                                                           int *flags, unsigned long long *mm) {
    typedef typename T::E E;
    const E *a = reinterpret_cast<const E *>(data);
    volatile int *vf = flags;
    unsigned long long lmin = ~0ull, lmax = 0;
    for (uint64_t c0 = (uint64_t)blockIdx.x * kDetectChunk; c0 < n;
         c0 += (uint64_t)gridDim.x * kDetectChunk) {
        if (!mm && __syncthreads_or(vf[0] == 0 && vf[1] == 0)) return;
        bool inc = true, dec = true;
        const uint64_t c1 = min(c0 + kDetectChunk, n);
        for (uint64_t i = c0 + threadIdx.x; i < c1; i += blockDim.x) {
            const E x = a[i];
            if (mm) {
                const unsigned long long r = T::rkey(x);
                lmin = min(lmin, r);
                lmax = max(lmax, r);
            }
            if (i + 1 < n) {
                typename T::K k0 = T::key(x), k1 = T::key(a[i + 1]);
                if (k1 < k0) inc = false;
                if (k0 < k1) dec = false;
            }
        }
        const int not_inc = __syncthreads_or(!inc);
        const int not_dec = __syncthreads_or(!dec);
        if (threadIdx.x == 0) {
            if (not_inc && vf[0]) flags[0] = 0;
            if (not_dec && vf[1]) flags[1] = 0;
        }
    }
    if (mm) {
        for (int o = 16; o > 0; o >>= 1) {
            lmin = min(lmin, __shfl_xor_sync(0xffffffffu, lmin, o));
            lmax = max(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMin(&mm[0], lmin);
            atomicMax(&mm[1], lmax);
        }
    }
}

template <class T>
__global__ void __launch_bounds__(256) k_reverse(unsigned char *data, uint64_t n,
                                                 const int *flags) {
    typedef typename T::E E;
    // reverse only an input that is non-increasing and not also non-decreasing
    if (!(flags[1] && !flags[0])) return;
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
template <>
__device__ __forceinline__ Key192 shfl_key<TQuartet>(Key192 k, int src) {
    Key192 r;
    r.a = __shfl_sync(0xffffffffu, k.a, src);
    r.b = __shfl_sync(0xffffffffu, k.b, src);
    r.c = __shfl_sync(0xffffffffu, k.c, src);
    return r;
}

// Bulk prefetch of [addr, addr + bytes) into L2 (both multiples of 16).
__device__ __forceinline__ void prefetch_l2(uint64_t addr, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(addr), "r"(bytes) : "memory");
}

// Copies one U-byte unit (U = 4, 8 or 16) from shared to global memory.
template <int U>
__device__ __forceinline__ void store_unit(unsigned char *dst, const unsigned char *src) {
    if (U == 16)
        *reinterpret_cast<uint4 *>(dst) = *reinterpret_cast<const uint4 *>(src);
    else if (U == 8)
        *reinterpret_cast<uint2 *>(dst) = *reinterpret_cast<const uint2 *>(src);
    else
        *reinterpret_cast<uint32_t *>(dst) = *reinterpret_cast<const uint32_t *>(src);
}

// Insertion sort of r[0..c) in shared memory (one thread).
template <class T>
__device__ __forceinline__ void insertion_sort(typename T::E *r, uint32_t c) {
    typedef typename T::E E;
    typedef typename T::K K;
    for (uint32_t i = 1; i < c; i++) {
        const E x = r[i];
        const K kx = T::key(x);
        uint32_t j = i;
        while (j > 0 && kx < T::key(r[j - 1])) {
            r[j] = r[j - 1];
            j--;
        }
        r[j] = x;
    }
}

// Sorts r[0..c), 2 <= c <= 4, in registers with the optimal 4-input
// network (0,1) (2,3) (0,2) (1,3) (1,2); a comparator touching position c
// or above is skipped, which leaves the 3- and 2-input networks.
template <class T>
__device__ __forceinline__ void sort_upto4(typename T::E *r, uint32_t c) {
    typedef typename T::E E;
    typedef typename T::K K;
    E x[4];
    K k[4];
#pragma unroll
    for (int i = 0; i < 4; i++) {
        x[i] = r[(uint32_t)i < c ? i : 0];
        k[i] = T::key(x[i]);
    }
    auto ce = [&](int i, int j) {
        if (k[j] < k[i]) {
            const E tx = x[i];
            x[i] = x[j];
            x[j] = tx;
            const K tk = k[i];
            k[i] = k[j];
            k[j] = tk;
        }
    };
    ce(0, 1);
    if (c > 3) ce(2, 3);
    if (c > 2) ce(0, 2);
    if (c > 3) ce(1, 3);
    if (c > 2) ce(1, 2);
#pragma unroll
    for (int i = 0; i < 4; i++)
        if ((uint32_t)i < c) r[i] = x[i];
}

// Sorts r[0..c), 5 <= c <= 8, in registers with Batcher's odd-even merge
// network for 8 inputs (19 comparators); as above, a comparator touching
// position c or above is skipped, which leaves a network for the first c.
template <class T>
__device__ __forceinline__ void sort_upto8(typename T::E *r, uint32_t c) {
    typedef typename T::E E;
    typedef typename T::K K;
    E x[8];
    K k[8];
#pragma unroll
    for (int i = 0; i < 8; i++) {
        x[i] = r[(uint32_t)i < c ? i : 0];
        k[i] = T::key(x[i]);
    }
    auto ce = [&](int i, int j) {
        if ((uint32_t)j < c && k[j] < k[i]) {
            const E tx = x[i];
            x[i] = x[j];
            x[j] = tx;
            const K tk = k[i];
            k[i] = k[j];
            k[j] = tk;
        }
    };
    ce(0, 1), ce(2, 3), ce(4, 5), ce(6, 7);
    ce(0, 2), ce(1, 3), ce(4, 6), ce(5, 7);
    ce(1, 2), ce(5, 6);
    ce(0, 4), ce(1, 5), ce(2, 6), ce(3, 7);
    ce(2, 4), ce(3, 5);
    ce(1, 2), ce(3, 4), ce(5, 6);
#pragma unroll
    for (int i = 0; i < 8; i++)
        if ((uint32_t)i < c) r[i] = x[i];
}

// Sorts each listed segment (segs[4i] = device byte address, segs[4i+1] = n
// <= smax, segs[4i+2..4i+3] = bounds lo <= hi of every element's radix key
// T::rkey, or lo > hi when not known) in place; the number of segments is
// *nsegs_dev if given, else nsegs_host.  One CTA per segment at a time; its
// bytes were prefetched into L2 while the CTA sorted its previous segment.
//
// The segment is staged into shared memory by one bulk copy; its radix key
// range is the given bounds (a bucket's splitters, or its radix digit) or,
// when none are known, the min/max of the staged keys.  A pass over a range
// [a0, a0+len) then counts an MSD radix digit of (key - min) (up to 2^DBITS
// digits, packed 16-bit counters; the offset itself when the range has
// that few values, else scaled to the digits), turns the counts into
// cursors, and scatters the range by digit from its global copy (which
// equals the shared one) into shared memory; afterwards the cursor of digit
// d is the end of its sub-bucket.  Sub-buckets of at most kBaseInsertion
// elements are finished in shared memory, one thread per sub-bucket (by a
// sorting network for up to 4, or up to 8 elements of at most 16 bytes,
// else insertion sort); those of at most kBaseSmall elements wait for one
// warp each once every larger range is done (equal keys skipped, few
// distinct keys peeled, others ranked); larger ones get another pass (with
// their own min/max).  Every pass writes its range back to global memory
// (coalesced), so the global copy of a pending range always matches the
// shared one.
//
// Two shapes share the code (BaseShape): one 1024-thread CTA per SM with
// 184 KiB of elements, and two 512-thread CTAs per SM with 88 KiB each, which
// take the segments that fit so that one CTA's loads and stores overlap the
// other's counting and scattering.  Each launch sorts the listed segments
// of its shape (base_goes_large).
template <int NT_, int BUF_, int MAXB_, int SSTK_>
struct BaseShape {
    static constexpr int NT = NT_;          // threads of a CTA
    static constexpr int BUF = BUF_;        // element buffer bytes
    static constexpr int MAXB = MAXB_;      // digit bits of the counter array
    static constexpr int SSTK = SSTK_;      // pending small ranges (>= BUF / 4 / 25)
    static constexpr int CTAS = 1024 / NT_;  // CTAs per SM
};
typedef BaseShape<1024, kBaseSmemBytes, kBaseDigitBits, kBaseSmallStack> BaseLarge;
typedef BaseShape<512, 88 * 1024, kBaseDigitBits - 1, 1024> BaseSmall;

// Whether a segment goes to the large shape: above the small shape's
// capacity, and also a segment of 4-byte keys whose known key range holds
// more than 2^13 and at most 2^14 values, when it is large enough for one
// exact pass there (one digit per key value among the large shape's 2^14
// digits; the small shape's 2^13 would put two values into each digit and
// leave their duplicates to be finished apart).
template <class T>
__device__ __forceinline__ bool base_goes_large(uint64_t n, uint64_t rlo, uint64_t rhi,
                                                uint64_t small_cap) {
    if (n > small_cap) return true;
    if (T::D > 4 || rlo > rhi || n <= (1ull << BaseSmall::MAXB)) return false;
    const uint64_t r = rhi - rlo;
    return r >= (1ull << BaseSmall::MAXB) && r < (1ull << BaseLarge::MAXB);
}

template <class T, class S>
__global__ void __launch_bounds__(S::NT, S::CTAS) k_base(const uint64_t *segs,
                                                         uint32_t nsegs_host,
                                                         const uint32_t *nsegs_dev, int *status,
                                                         uint64_t n_lo, uint64_t n_hi) {
    typedef typename T::E E;
    typedef typename T::K K;
    constexpr int kBaseThreads = S::NT;
    // Digits per pass: about two elements per digit for keys up to 8 bytes,
    // one for wider records (whose insertion-sort moves cost more), at most
    // 2^MAXB digits for 4-byte keys and half that otherwise, which leaves
    // the upper half of the counter words to the list of mid-size
    // sub-buckets (measured optima: 2^13 digits in the large shape, 2^12 in
    // the small one) -- unless one digit per key value fits in 2^MAXB
    // digits and at most twice that many: then the pass is final (no
    // finishing sorts)
    constexpr int DBITS = T::D <= 4 ? S::MAXB : S::MAXB - 1;
    constexpr uint32_t kPerDigitLog = T::D <= 8 ? 1u : 0u;
    constexpr int ND = 1 << S::MAXB;
    constexpr int NB = T::D <= 8 ? 8 : (T::D <= 16 ? 4 : (T::D <= 32 ? 2 : 1));  // in flight per thread
    constexpr int U = T::D % 16 == 0 ? 16 : (T::D % 8 == 0 ? 8 : 4);  // copy-out unit
    extern __shared__ __align__(16) unsigned char smem[];
    // layout: buf (BUF + 16 bytes: a segment is placed at its global
    // address modulo 16, so that a bulk copy moves its aligned interior) |
    // stk | sstk | cur (ND/2 words, two 16-bit counters each) | wtmp.
    // Ranges are < 2^16 elements, so 16-bit counters and cursors suffice.
    // Digits 2w and 2w + 1 share word w.
    uint32_t *stk = reinterpret_cast<uint32_t *>(smem + S::BUF + 16);  // (a0 << 16) | len
    uint32_t *sstk = stk + kBaseStack;                            // small ranges
    uint32_t *cur = sstk + S::SSTK;                               // ND / 2
    uint32_t *wtmp = cur + ND / 2;                                         // 34
    __shared__ unsigned long long red[2][32];
    __shared__ uint32_t sp, ssp, sh_top, sh_nmid;
    __shared__ __align__(8) uint64_t sh_bar;  // completion of a segment's bulk copy
    uint32_t parity = 0;
    // sorting networks and the mid-size list for keys up to 32 bytes
    constexpr bool kNetwork = T::D <= 32;
    constexpr uint32_t kNoRange = 0xFFFFFFFFu;  // no range has a0 = len = 65535
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = kBaseThreads / 32;
    if (tid == 0) {
        mbar_init(&sh_bar, 1);
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    }
    __syncthreads();

    // CTA-wide min and max of per-thread values (all threads call it)
    auto minmax = [&](unsigned long long lmin, unsigned long long lmax, uint64_t &gmn,
                      uint64_t &gmx) {
        for (int o = 16; o > 0; o >>= 1) {
            lmin = min(lmin, __shfl_xor_sync(0xffffffffu, lmin, o));
            lmax = max(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
        }
        if (lane == 0) {
            red[0][warp] = lmin;
            red[1][warp] = lmax;
        }
        __syncthreads();
        unsigned long long a = red[0][0], b = red[1][0];
        for (int w = 1; w < NW; w++) {
            a = min(a, red[0][w]);
            b = max(b, red[1][w]);
        }
        __syncthreads();
        gmn = a;
        gmx = b;
    };
    auto word = [](uint32_t d) -> uint32_t { return d >> 1; };
    // end of digit d's sub-bucket once the scatter has run
    auto dend = [&](uint32_t d) -> uint32_t { return (cur[word(d)] >> (16 * (d & 1))) & 0xFFFFu; };

    const uint32_t nsegs = nsegs_dev ? *nsegs_dev : nsegs_host;
    // the small shape's launch takes n in (n_lo = 0, n_hi = its capacity],
    // the large one's (n_lo = that capacity, n_hi = ~0), both refined by
    // base_goes_large
    constexpr bool kLarge = S::NT == BaseLarge::NT;
    const uint64_t small_cap = kLarge ? n_lo : n_hi;
    for (uint32_t si = blockIdx.x; si < nsegs; si += gridDim.x) {
        const uint64_t addr = segs[4 * si], n = segs[4 * si + 1];
        const uint64_t rlo = segs[4 * si + 2], rhi = segs[4 * si + 3];
        if (base_goes_large<T>(n, rlo, rhi, small_cap) != kLarge) continue;  // the other shape's
        E *g = reinterpret_cast<E *>(addr);
        E *buf = reinterpret_cast<E *>(smem + (addr & 15));
        if (tid == 0 && si + gridDim.x < nsegs) {
            // the CTA's next segment streams into L2 while this one is sorted
            const uint64_t na = segs[4 * (si + gridDim.x)], nn = segs[4 * (si + gridDim.x) + 1];
            const uint64_t lo = (na + 15) & ~15ull, hi = (na + nn * T::D) & ~15ull;
            if (base_goes_large<T>(nn, segs[4 * (si + gridDim.x) + 2], segs[4 * (si + gridDim.x) + 3],
                                   small_cap) == kLarge &&
                hi > lo)
                prefetch_l2(lo, (uint32_t)(hi - lo));
        }
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
        // stage the segment into shared memory through registers, with the
        // min / max of the high radix-key word
        // the segment arrives by one bulk copy (its unaligned ends by 4-byte
        // copies), bounded wait; its key range is the given bounds, or the
        // min / max of its leading key word when none are known
        uint64_t seg_mn = rlo, seg_mx = rhi;
        tile_load(reinterpret_cast<unsigned char *>(buf),
                  reinterpret_cast<const unsigned char *>(g), (uint32_t)n * T::D, &sh_bar);
        const bool landed = mbar_wait_bounded(&sh_bar, parity, kBaseSpin);
        parity ^= 1;
        cp_async_wait_all();
        if (__syncthreads_or(!landed)) {
            if (tid == 0) set_status(status, IPSGPU_E_TIMEOUT);
            mbar_wait_bounded(&sh_bar, parity ^ 1, kBaseSpin);
            return;
        }
        if (rlo > rhi) {
            unsigned long long lmin = ~0ull, lmax = 0;
            for (uint32_t i = tid; i < n; i += kBaseThreads) {
                const unsigned long long v = T::rkey(buf[i]);
                lmin = min(lmin, v);
                lmax = max(lmax, v);
            }
            minmax(lmin, lmax, seg_mn, seg_mx);
        }
        if (tid == 0) {
            sp = 1;
            ssp = 0;
            sh_nmid = 0;
            stk[0] = (uint32_t)n;
        }
        bool first = true;
        while (true) {
            // thread 0 pops the next pending range and publishes it between
            // two barriers, so every thread sees the same range (or the end)
            // whichever way the previous pass ended
            __syncthreads();
            if (tid == 0) {
                if (sp > kBaseStack) sp = kBaseStack;  // pushes past the stack were dropped
                sh_top = sp ? stk[sp - 1] : kNoRange;
                if (sp) sp--;
                sh_nmid = 0;  // the last pass's list has been read
            }
            __syncthreads();
            const uint32_t top = sh_top;
            if (top == kNoRange) break;
            // a range is packed as (a0 << 16) | len; both are < 2^16 because
            // a segment holds at most kBaseSmemBytes / 4 < 2^16 elements
            const uint32_t a0 = top >> 16, len = top & 0xFFFFu;
            // min / max of the radix key over the range: of its leading
            // word, or, for keys wider than 64 bits, of the first word that
            // is not constant over the range
            int mode = 0;  // the key word the pass sorts by
            uint64_t mn = 0, rng = 0;
            for (int pass = 0; pass < T::kKeyWords; pass++) {
                uint64_t gmn, gmx;
                if (first && pass == 0) {
                    gmn = seg_mn;
                    gmx = seg_mx;
                } else {
                    unsigned long long lmin = ~0ull, lmax = 0;
                    for (uint32_t i = tid; i < len; i += kBaseThreads) {
                        const uint64_t v = rk_word<T>(buf[a0 + i], pass);
                        lmin = min(lmin, (unsigned long long)v);
                        lmax = max(lmax, (unsigned long long)v);
                    }
                    minmax(lmin, lmax, gmn, gmx);
                }
                mode = pass;
                mn = gmn;
                rng = gmx - gmn;
                if (rng != 0) break;
            }
            first = false;
            if (rng == 0) continue;  // all keys equal: the range is final
            const uint32_t nbits = 64 - __clzll((long long)rng);
            uint32_t want = 1;
            while (want < (uint32_t)DBITS && ((1u << kPerDigitLog) << want) < len) want++;
            const uint32_t dbits =
                (nbits <= (uint32_t)S::MAXB && nbits <= want + 1) ? nbits : min(nbits, want);
            const uint32_t nd = 1u << dbits;
            const uint32_t nw = (nd + 1) >> 1;  // counter words in use
            // A digit is the whole offset v - mn when the range has at most
            // 2^dbits values; otherwise the offset scaled to [0, nd): its top
            // 32 bits (below bit nbits) times m / 2^32, m = nd 2^32 / (top
            // of the range + 1) -- nondecreasing in v, below nd, and spread
            // over all nd digits (a power-of-two shift would leave up to
            // half of them empty and crowd the rest)
            const bool whole = nbits == dbits;
            const uint32_t s2 = nbits > 32 ? nbits - 32 : 0u;
            const uint32_t m =
                whole ? 0u
                      : (uint32_t)(((uint64_t)nd << 32) / ((uint64_t)(uint32_t)(rng >> s2) + 1));
            auto digit = [&](uint64_t v) -> uint32_t {
                return whole ? (uint32_t)(v - mn) : __umulhi((uint32_t)((v - mn) >> s2), m);
            };
            // with whole offsets in the last word (the words before it are
            // constant) each sub-bucket holds one key, so it is final
            const bool exact = whole && mode == T::kKeyWords - 1;
            for (uint32_t w = tid; w < nw; w += kBaseThreads) cur[w] = 0;
            __syncthreads();
            for (uint32_t i = tid; i < len; i += kBaseThreads) {
                const uint64_t v = rk_word<T>(buf[a0 + i], mode);
                const uint32_t d = digit(v);
                atomicAdd(&cur[word(d)], 1u << (16 * (d & 1)));
            }
            __syncthreads();
            {
                // exclusive scan of the 16-bit counts; each thread owns a
                // run of consecutive counter words of the nd digits in use,
                // sums it, and after the CTA-wide scan rewrites it as cursors
                const uint32_t wpt = (nw + kBaseThreads - 1) / kBaseThreads;
                const uint32_t w0 = min(nw, tid * wpt), w1 = min(nw, w0 + wpt);
                uint32_t sum = 0;
                for (uint32_t w = w0; w < w1; w++) {
                    const uint32_t c2 = cur[w];
                    sum += (c2 & 0xFFFFu) + (c2 >> 16);
                }
                uint32_t x = sum;
                for (int o = 1; o < 32; o <<= 1) {
                    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                    if (lane >= o) x += y;
                }
                if (lane == 31) wtmp[warp] = x;
                __syncthreads();
                if (warp == 0) {
                    uint32_t w = lane < NW ? wtmp[lane] : 0u, v = w;
                    for (int o = 1; o < 32; o <<= 1) {
                        uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
                        if (lane >= o) v += y;
                    }
                    if (lane < NW) wtmp[lane] = v - w;
                }
                __syncthreads();
                uint32_t run = wtmp[warp] + x - sum;
                for (uint32_t w = w0; w < w1; w++) {
                    const uint32_t c2 = cur[w];
                    const uint32_t o0 = run, o1 = run + (c2 & 0xFFFFu);
                    run = o1 + (c2 >> 16);
                    cur[w] = o0 | (o1 << 16);
                }
            }
            __syncthreads();
            // scatter by digit, reading the range's global copy in batches;
            // each cursor ends at the end of its digit's sub-bucket
            for (uint32_t i0 = 0; i0 < len; i0 += NB * kBaseThreads) {
                E x[NB];
#pragma unroll
                for (int q = 0; q < NB; q++) {
                    const uint32_t i = i0 + q * kBaseThreads + tid;
                    if (i < len) x[q] = g[a0 + i];
                }
#pragma unroll
                for (int q = 0; q < NB; q++) {
                    const uint32_t i = i0 + q * kBaseThreads + tid;
                    if (i < len) {
                        const uint64_t v = rk_word<T>(x[q], mode);
                        const uint32_t d = digit(v);
                        const uint32_t h = 16 * (d & 1);
                        const uint32_t p = (atomicAdd(&cur[word(d)], 1u << h) >> h) & 0xFFFFu;
                        buf[a0 + p] = x[q];
                    }
                }
            }
            __syncthreads();
            // per sub-bucket (one thread each): a large one gets another
            // pass or waits for a warp; one of 2..4 elements is sorted by a
            // 5-comparator network in registers (comparators predicated on
            // the size, so the warp does not diverge on it); one of 5..24
            // elements goes to a list (the counter words this pass leaves
            // unused) that threads take one entry each afterwards, so that
            // no warp waits for its lanes' longest insertion sort; when the
            // list is full (always for 4-byte keys, whose digits take every
            // counter word), or for records, it is sorted right away: by the
            // 8-input network up to 8 elements of at most 16 bytes (keys
            // with many duplicates fill such sub-buckets), else by insertion
            // sort
            uint32_t *mid = cur + nw;
            const uint32_t mid_cap = (uint32_t)(ND / 2) - nw;
            for (uint32_t d = tid; d < nd && !exact; d += kBaseThreads) {
                const uint32_t lo = d ? dend(d - 1) : 0u, c = dend(d) - lo;
                if (c > kBaseSmall) {
                    uint32_t q = atomicAdd(&sp, 1u);
                    if (q < kBaseStack)
                        stk[q] = ((a0 + lo) << 16) | c;
                    else
                        set_status(status, IPSGPU_E_INTERNAL);
                } else if (c > kBaseInsertion) {
                    uint32_t q = atomicAdd(&ssp, 1u);
                    if (q < (uint32_t)S::SSTK)
                        sstk[q] = ((a0 + lo) << 16) | c;
                    else
                        set_status(status, IPSGPU_E_INTERNAL);
                } else if (kNetwork && c <= 4) {
                    if (c > 1) sort_upto4<T>(buf + a0 + lo, c);
                } else if (c > 1) {
                    const uint32_t q = kNetwork && mid_cap ? atomicAdd(&sh_nmid, 1u) : mid_cap;
                    if (q < mid_cap) {
                        mid[q] = (lo << 16) | c;
                    } else {
                        bool done = false;
                        if constexpr (T::D <= 16) {
                            if (c <= 8) {
                                sort_upto8<T>(buf + a0 + lo, c);
                                done = true;
                            }
                        }
                        if (!done) insertion_sort<T>(buf + a0 + lo, c);
                    }
                }
            }
            if (kNetwork) {
                __syncthreads();
                const uint32_t nmid = min(sh_nmid, mid_cap);
                for (uint32_t q = tid; q < nmid; q += kBaseThreads) {
                    // up to 8 elements of at most 16 bytes: a network in
                    // registers, whose lanes run in step; else insertion sort
                    const uint32_t lo = mid[q] >> 16, c = mid[q] & 0xFFFFu;
                    if constexpr (T::D <= 16) {
                        if (c <= 8) {
                            sort_upto8<T>(buf + a0 + lo, c);
                            continue;
                        }
                    }
                    insertion_sort<T>(buf + a0 + lo, c);
                }
            }
            __syncthreads();
            // the range back to global memory, coalesced: final where the
            // sub-buckets were small, grouped by digit where they were large
            {
                const uint32_t units = (uint32_t)((uint64_t)len * T::D / U);
                const unsigned char *src = reinterpret_cast<const unsigned char *>(buf + a0);
                unsigned char *dst = reinterpret_cast<unsigned char *>(g + a0);
                for (uint32_t u = tid; u < units; u += kBaseThreads)
                    store_unit<U>(dst + (size_t)u * U, src + (size_t)u * U);
            }
        }
        // the small ranges, one warp each: a range of equal keys is final;
        // a range of at most kBasePeel distinct keys (duplicates) is peeled
        // smallest key first, each key's elements to the next positions in
        // their order; otherwise each element goes to its rank within the
        // range (ties by position).  Either way straight to global memory.
        // Shared memory holds the range as the last pass grouped it, like
        // its global copy.
        const uint32_t nsmall = min(ssp, (uint32_t)S::SSTK);
        for (uint32_t r = warp; r < nsmall; r += NW) {
            const uint32_t top = sstk[r];
            const uint32_t a0 = top >> 16, c = top & 0xFFFFu;
            unsigned long long mn[T::kKeyWords], mx[T::kKeyWords];
#pragma unroll
            for (int w = 0; w < T::kKeyWords; w++) {
                mn[w] = ~0ull;
                mx[w] = 0;
            }
            for (uint32_t p = lane; p < c; p += 32) {
#pragma unroll
                for (int w = 0; w < T::kKeyWords; w++) {
                    const unsigned long long v = rk_word<T>(buf[a0 + p], w);
                    mn[w] = min(mn[w], v);
                    mx[w] = max(mx[w], v);
                }
            }
            bool all_equal = true;
#pragma unroll
            for (int w = 0; w < T::kKeyWords; w++) {
                for (int o = 16; o > 0; o >>= 1) {
                    mn[w] = min(mn[w], __shfl_xor_sync(0xffffffffu, mn[w], o));
                    mx[w] = max(mx[w], __shfl_xor_sync(0xffffffffu, mx[w], o));
                }
                all_equal = all_equal && mn[w] == mx[w];
            }
            if (all_equal) continue;  // all keys equal
            uint32_t done = 0;  // elements placed (warp-uniform)
            K last = T::max_key();
            for (int it = 0; it < kBasePeel && done < c; it++) {
                // the smallest key above the last one peeled
                K v = T::max_key();
                for (uint32_t p = lane; p < c; p += 32) {
                    const K k = T::key(buf[a0 + p]);
                    if ((it == 0 || last < k) && k < v) v = k;
                }
                for (int o = 16; o > 0; o >>= 1) {
                    const K ov = shfl_key<T>(v, lane ^ o);
                    if (ov < v) v = ov;
                }
                for (uint32_t p0 = 0; p0 < c; p0 += 32) {
                    const uint32_t p = p0 + (uint32_t)lane;
                    bool eq = false;
                    if (p < c) {
                        const K k = T::key(buf[a0 + p]);
                        eq = !(k < v) && !(v < k);
                    }
                    const uint32_t m = __ballot_sync(0xffffffffu, eq);
                    if (eq) g[a0 + done + __popc(m & ((1u << lane) - 1u))] = buf[a0 + p];
                    done += __popc(m);
                }
                last = v;
            }
            if (done >= c) continue;  // every key peeled
            for (uint32_t p = lane; p < c; p += 32) {
                const E x = buf[a0 + p];
                const K kx = T::key(x);
                uint32_t rank = 0;
                for (uint32_t q = 0; q < c; q++) {
                    const K kq = T::key(buf[a0 + q]);
                    rank += (kq < kx || (!(kx < kq) && q < p)) ? 1u : 0u;
                }
                g[a0 + rank] = x;
            }
        }
        __syncthreads();
    }
}

template <class S>
inline size_t base_smem_bytes() {
    return S::BUF + 16 + sizeof(uint32_t) * (kBaseStack + S::SSTK) +
           sizeof(uint32_t) * ((1 << S::MAXB) / 2 + 34) + 16;
}

}  // namespace ipsgpu

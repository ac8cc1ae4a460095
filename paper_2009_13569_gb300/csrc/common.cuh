// common.cuh -- element traits, device helpers and the layouts shared by the
// kernels of one partitioning level (Sec. 3.1 of Axtmann et al.).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ipsgpu.h"

namespace ipsgpu {

// ---------------------------------------------------------------- limits
constexpr int kMaxClasses = 256;      // buckets per level incl. equality ones
constexpr uint32_t kMaxBlockBytes = 2048;  // a block, held by one warp in registers
// sample keys sorted in one CTA: the largest power of two <= 16384 whose
// keys fit in 192 KiB (the bitonic sort pads the sample to a power of two):
// 16384 keys of 4 or 8 bytes, 8192 of 16 or 24 bytes
template <class K>
constexpr uint32_t max_sort_sample() {
    uint32_t m = 16384u;
    while (m > 1 && (uint64_t)m * sizeof(K) > 192u * 1024) m >>= 1;
    return m;
}
constexpr uint32_t kRBias = 1u << 30; // bias of the read pointer field
constexpr int kBaseSmemBytes = 184 * 1024;  // element buffer of the base case

// ------------------------------------------------------------ key types
// Rec100 keys: bytes 0..7 big-endian in hi, bytes 8..9 big-endian in lo.
struct Key80 {
    uint64_t hi;
    uint32_t lo;
};
__host__ __device__ inline bool operator<(const Key80 &a, const Key80 &b) {
    return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}
__host__ __device__ inline bool operator==(const Key80 &a, const Key80 &b) {
    return a.hi == b.hi && a.lo == b.lo;
}

// Quartet keys: three u64 words compared lexicographically (Sec. 6)
struct Key192 {
    uint64_t a, b, c;
};
__host__ __device__ inline bool operator<(const Key192 &x, const Key192 &y) {
    return x.a != y.a ? x.a < y.a : (x.b != y.b ? x.b < y.b : x.c < y.c);
}
__host__ __device__ inline bool operator==(const Key192 &x, const Key192 &y) {
    return x.a == y.a && x.b == y.b && x.c == y.c;
}

struct PairElem {
    uint64_t k, v;
};
// 16-byte aligned so that an element moves as two 16-byte accesses
struct __align__(16) QuartetElem {
    uint64_t a, b, c, v;
};
struct Rec100Elem {
    uint32_t w[25];
};

// Element traits.  E: element storage, K: key, D: bytes, key(): order key,
// rkey(): the key's leading 64-bit word (radix key of the base case and of
// the start-node table), kKeyWords: 64-bit words the base case's radix
// passes walk through (rk_word<T>(e, w), w < kKeyWords), kHeadLanes: lanes of a
// warp-held block (16 bytes each) that hold its first element's key,
// head(): that element from lane 0's (and lane 1's) 16 bytes.
struct TU32 {
    typedef uint32_t E;
    typedef uint32_t K;
    static constexpr int D = 4;
    static constexpr bool kRadix = true;
    static constexpr int kKeyWords = 1;
    static constexpr int kHeadLanes = 1;
    __device__ static K key(const E &e) { return e; }
    __device__ static uint64_t rkey(const E &e) { return e; }
    __device__ static K max_key() { return 0xFFFFFFFFu; }
    __device__ static E head(uint4 h) { return h.x; }
};
struct TU64 {
    typedef uint64_t E;
    typedef uint64_t K;
    static constexpr int D = 8;
    static constexpr bool kRadix = true;
    static constexpr int kKeyWords = 1;
    static constexpr int kHeadLanes = 1;
    __device__ static K key(const E &e) { return e; }
    __device__ static uint64_t rkey(const E &e) { return e; }
    __device__ static K max_key() { return ~0ull; }
    __device__ static E head(uint4 h) { return (uint64_t)h.x | ((uint64_t)h.y << 32); }
};
// f64: order key = (b>>63) ? ~b : b | 2^63 on the IEEE bits
struct TF64 {
    typedef uint64_t E;
    typedef uint64_t K;
    static constexpr int D = 8;
    static constexpr bool kRadix = false;
    static constexpr int kKeyWords = 1;
    static constexpr int kHeadLanes = 1;
    __device__ static K key(const E &e) {
        return (e >> 63) ? ~e : (e | 0x8000000000000000ull);
    }
    __device__ static uint64_t rkey(const E &e) { return key(e); }
    __device__ static K max_key() { return ~0ull; }
    __device__ static E head(uint4 h) { return (uint64_t)h.x | ((uint64_t)h.y << 32); }
};
struct TPair {
    typedef PairElem E;
    typedef uint64_t K;
    static constexpr int D = 16;
    static constexpr bool kRadix = true;
    static constexpr int kKeyWords = 1;
    static constexpr int kHeadLanes = 1;
    __device__ static K key(const E &e) { return e.k; }
    __device__ static uint64_t rkey(const E &e) { return e.k; }
    __device__ static K max_key() { return ~0ull; }
    __device__ static E head(uint4 h) {
        E e;
        e.k = (uint64_t)h.x | ((uint64_t)h.y << 32);
        e.v = (uint64_t)h.z | ((uint64_t)h.w << 32);
        return e;
    }
};
struct TRec100 {
    typedef Rec100Elem E;
    typedef Key80 K;
    static constexpr int D = 100;
    static constexpr bool kRadix = false;
    static constexpr int kKeyWords = 2;
    static constexpr int kHeadLanes = 1;
    // bytes 0..3 of a record are w[0] little-endian, so byte-swapping w[0]
    // and w[1] gives bytes 0..7 in big-endian (lexicographic) order
    __device__ static K key_words(uint32_t w0, uint32_t w1, uint32_t w2) {
        K k;
        k.hi = ((uint64_t)__byte_perm(w0, 0, 0x0123) << 32) | __byte_perm(w1, 0, 0x0123);
        k.lo = ((w2 & 0xFFu) << 8) | ((w2 >> 8) & 0xFFu);
        return k;
    }
    __device__ static K key(const E &e) { return key_words(e.w[0], e.w[1], e.w[2]); }
    __device__ static uint64_t rkey(const E &e) { return key(e).hi; }
    __device__ static K max_key() {
        K k;
        k.hi = ~0ull;
        k.lo = 0xFFFFFFFFu;
        return k;
    }
    // only the first 16 bytes (the key and 6 payload bytes) are meaningful
    __device__ static E head(uint4 h) {
        E e;
        e.w[0] = h.x;
        e.w[1] = h.y;
        e.w[2] = h.z;
        e.w[3] = h.w;
        return e;
    }
};

struct TQuartet {
    typedef QuartetElem E;
    typedef Key192 K;
    static constexpr int D = 32;
    static constexpr bool kRadix = false;
    static constexpr int kKeyWords = 3;
    static constexpr int kHeadLanes = 2;
    __device__ static K key(const E &e) {
        K k;
        k.a = e.a;
        k.b = e.b;
        k.c = e.c;
        return k;
    }
    __device__ static uint64_t rkey(const E &e) { return e.a; }
    __device__ static K max_key() {
        K k;
        k.a = k.b = k.c = ~0ull;
        return k;
    }
    __device__ static E head2(uint4 h0, uint4 h1) {
        E e;
        e.a = (uint64_t)h0.x | ((uint64_t)h0.y << 32);
        e.b = (uint64_t)h0.z | ((uint64_t)h0.w << 32);
        e.c = (uint64_t)h1.x | ((uint64_t)h1.y << 32);
        e.v = (uint64_t)h1.z | ((uint64_t)h1.w << 32);
        return e;
    }
};

// The leading 64-bit word of a key (T::rkey of an element with that key),
// and the largest value it takes.
template <class T>
__device__ __forceinline__ uint64_t rk_of_key(const typename T::K &k) {
    return (uint64_t)k;
}
template <>
__device__ __forceinline__ uint64_t rk_of_key<TRec100>(const Key80 &k) {
    return k.hi;
}
template <>
__device__ __forceinline__ uint64_t rk_of_key<TQuartet>(const Key192 &k) {
    return k.a;
}
template <class T>
__host__ __device__ constexpr uint64_t rk_max() {
    return sizeof(typename T::K) == 4 ? 0xFFFFFFFFull : ~0ull;
}

// The first element of a block held by a warp, 16 bytes per lane (lane 0's
// bytes, and lane 1's where the key reaches past them), broadcast: every
// lane calls it and gets the element.
__device__ __forceinline__ uint4 shfl_uint4(const uint4 &r, int src) {
    uint4 x;
    x.x = __shfl_sync(0xffffffffu, r.x, src);
    x.y = __shfl_sync(0xffffffffu, r.y, src);
    x.z = __shfl_sync(0xffffffffu, r.z, src);
    x.w = __shfl_sync(0xffffffffu, r.w, src);
    return x;
}
template <class T>
__device__ __forceinline__ typename T::E block_head(const uint4 &r) {
    if constexpr (T::kHeadLanes == 2)
        return T::head2(shfl_uint4(r, 0), shfl_uint4(r, 1));
    else
        return T::head(shfl_uint4(r, 0));
}

// ------------------------------------------------------------ level layouts
// Planned description of one segment partitioned in a level launch (written
// by the host planner, or on the device for the segmented batch).
struct SegDesc {
    uint64_t addr;       // device byte address of the segment's first element
    uint64_t n;          // elements
    uint32_t b;          // block size in elements
    uint32_t C;          // class budget (power of two <= 256): bounds B
    uint32_t stripe0;    // first stripe of the segment
    uint32_t nstripes;
    uint32_t cta0;       // first block-permutation CTA of the segment
    uint32_t ncta;
    uint64_t stage_off;  // arena bytes: cleanup staging (C blocks), then the overflow block
    uint64_t arr_off;    // state-arena bytes: per-class arrays (SegArrays)
    uint64_t key_off;    // key-arena bytes: tree[C] then splitters[C]
    uint32_t cls0;       // first (segment, class) work item: prefix sum of C
    uint32_t mode;       // 0: sample splitters, 1: given splitters, 2: radix
    uint32_t radix_shift;
    uint32_t radix_bits;
    uint32_t nsplit;     // given splitters (mode 1)
    uint32_t eq_given;
    uint32_t cnt0;       // first per-class count entry of the segment's stripes
    uint32_t part0;      // balanced waves: classification part of its first stripe
    uint64_t gblk0;      // balanced waves: first block in the wave's block order
    uint64_t rlo, rhi;   // every element's T::rkey lies in [rlo, rhi] (rlo > rhi: not known)
};

// Per-stripe plan and outputs.
struct StripeDesc {
    uint32_t seg;
    uint32_t blk0;       // first block of the stripe within its segment
    uint32_t nblk;       // blocks (the last one may be partial)
    uint32_t cnt_off;    // first entry of the stripe's per-class counts
    uint64_t left_off;   // arena bytes: leftover buffer blocks (C blocks)
};

// Device-computed header of a segment during a level.
struct SegState {
    uint32_t K, B, logK, eq;
    uint32_t nslots;       // ceil(n / b)
    uint32_t nfull_slots;  // floor(n / b)
    uint32_t ovf_used;     // 1 if a block was written to the overflow block
    uint32_t pad;
};

// Per-class arrays of a segment, C entries each, in the state arena:
//   u64 bucket_begin[C+1] | u64 ptr[C] | u32 readers[C] | u32 full[C] |
//   u32 dlm[C+1]
// ptr[i] packs the write pointer w_i (high half) and the exclusive read
// pointer r_i + 1 + kRBias (low half); dlm[i] is the delimiter (in blocks).
struct SegArrays {
    uint64_t *bb;
    unsigned long long *ptr;
    uint32_t *readers;
    uint32_t *full;
    uint32_t *dlm;
};
__host__ __device__ inline uint64_t seg_arrays_bytes(uint32_t C) {
    return ((uint64_t)28 * C + 12 + 15) & ~(uint64_t)15;
}
__device__ inline SegArrays seg_arrays(unsigned char *sarr, const SegDesc &sd) {
    unsigned char *p = sarr + sd.arr_off;
    SegArrays r;
    r.bb = reinterpret_cast<uint64_t *>(p);
    r.ptr = reinterpret_cast<unsigned long long *>(p + 8 * (sd.C + 1));
    r.readers = reinterpret_cast<uint32_t *>(p + 8 * (sd.C + 1) + 8 * sd.C);
    r.full = r.readers + sd.C;
    r.dlm = r.full + sd.C;
    return r;
}

struct Move {
    uint32_t seg;
    uint32_t src, dst, len;  // block indices within the segment
};

// Work counts of a level when they live in device memory (segmented batch);
// with cnt == nullptr the host-provided values in LevelArgs are used.
struct LevelCounts {
    uint32_t nseg, nstripe, ncta, ncls;
    uint32_t balanced;  // stripes are grouped into parts, one per classify CTA
    uint32_t pad;
};

struct LevelArgs {
    unsigned char *data;
    const SegDesc *seg;
    SegState *st;
    unsigned char *sarr;      // state arena (SegArrays)
    unsigned char *keys;      // key arena (tree, splitters)
    const unsigned char *given_spl;  // mode 1: user splitters (elements)
    const StripeDesc *stripe;
    uint32_t *scount;         // count arena: per stripe, C entries
    uint32_t *sfull;          // [nstripe] full blocks written by the stripe
    unsigned char *arena;     // leftovers, staging, overflow blocks
    Move *moves;
    uint32_t *nmoves;
    uint32_t move_cap;
    int *status;
    uint32_t nseg, nstripe, ncta, ncls;
    const LevelCounts *cnt;
    const uint32_t *cta_seg;
    const uint32_t *stripe_first;  // balanced waves: first stripe of each part
    uint32_t spin_limit;
    uint32_t tree_only;       // classification walks every element from the tree's root
    uint64_t seed;
    float alpha_scale;
    uint32_t pad2;
};

__device__ inline uint32_t lv_nseg(const LevelArgs &a) { return a.cnt ? a.cnt->nseg : a.nseg; }
__device__ inline uint32_t lv_nstripe(const LevelArgs &a) {
    return a.cnt ? a.cnt->nstripe : a.nstripe;
}
__device__ inline uint32_t lv_ncta(const LevelArgs &a) { return a.cnt ? a.cnt->ncta : a.ncta; }
__device__ inline uint32_t lv_ncls(const LevelArgs &a) { return a.cnt ? a.cnt->ncls : a.ncls; }

// ------------------------------------------------------------ helpers
__device__ inline void set_status(int *status, int code) {
    atomicCAS(status, 0, code);
}

__device__ inline uint64_t splitmix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

__host__ __device__ inline uint32_t ilog2_floor(uint64_t x) {
    uint32_t l = 0;
    while ((x >> l) > 1) l++;
    return l;
}

// Classification of one key (Sec. 2, refined branchless decision tree):
// descend i <- 2i + [tree_i < e] from the root for log2 K steps, leaf i - K;
// with equality buckets the class is 2i + 1 - [e < s_i].
template <class K>
__device__ __forceinline__ uint32_t classify_key(const K &e, const K *tree, const K *spl,
                                                 uint32_t logK, bool eq) {
    uint32_t i = 1;
    for (uint32_t l = 0; l < logK; l++) i = 2 * i + (tree[i] < e ? 1u : 0u);
    i -= (1u << logK);
    if (eq) i = 2 * i + 1 - (e < spl[i] ? 1u : 0u);
    return i;
}

// CTA-wide exclusive scan of cnt[0..N) into out[0..N); returns the total.
// All threads must call it; blockDim.x must be a multiple of 32.
template <typename T>
__device__ T cta_exclusive_scan(const T *cnt, T *out, int N, T *warp_tmp) {
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int per = (N + nthr - 1) / nthr;
    const int lo = min(N, tid * per), hi = min(N, lo + per);
    T s = 0;
    for (int i = lo; i < hi; i++) s += cnt[i];
    // inclusive warp scan of s
    T x = s;
    const int lane = tid & 31, warp = tid >> 5;
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tmp[warp] = x;
    __syncthreads();
    const int nw = nthr >> 5;
    if (warp == 0) {
        T w = lane < nw ? warp_tmp[lane] : (T)0;
        T v = w;
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += y;
        }
        if (lane < nw) warp_tmp[lane] = v - w;  // exclusive warp offsets
        if (lane == 31) warp_tmp[32] = v;        // total
    }
    __syncthreads();
    T run = warp_tmp[warp] + x - s;
    for (int i = lo; i < hi; i++) {
        T c = cnt[i];
        out[i] = run;
        run += c;
    }
    T total = warp_tmp[32];
    __syncthreads();
    return total;
}

// Bounded spin on a 32-bit device word: waits until *p == want or the
// iteration budget is spent.  Returns true on success.  On timeout the caller
// records IPSGPU_E_TIMEOUT and returns without touching shared data.
__device__ inline bool bounded_wait_eq(const volatile uint32_t *p, uint32_t want,
                                       uint32_t limit) {
    for (uint32_t it = 0; it < limit; it++) {
        if (*p == want) return true;
        __nanosleep(64);
    }
    return *p == want;
}

// ---------------------------------------------------- TMA bulk copies
// One-dimensional bulk copy global -> shared completed on an mbarrier
// (cp.async.bulk with complete_tx).  Both addresses and the size must be
// multiples of 16 bytes.
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for phase `parity` of an mbarrier; false if it gave up.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint32_t limit) {
    for (uint32_t it = 0; it < limit; it++)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void bulk_load(void *dst_smem, const void *src, uint32_t bytes,
                                          uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::
            "r"(smem_addr(dst_smem)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

}  // namespace ipsgpu

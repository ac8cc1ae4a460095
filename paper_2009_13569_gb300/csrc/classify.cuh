// classify.cuh -- classification with buffer blocks (Sec. 3.1.2 of Axtmann et
// al.), the first half of every partitioning level.
//
// One CTA owns one stripe (a run of whole blocks of its segment).  The stripe
// is read tile by tile; the next tile streams into shared memory with
// cp.async while the current one is processed:
//   [B] every thread classifies its elements and takes a rank inside its
//       class with a shared-memory atomic (one per warp when all its lanes
//       share a class);
//   [C] per class, the buffer blocks that fill up in this tile get slots at
//       the front of the stripe (an atomic on the stripe's block counter:
//       the order of full blocks in a stripe is free);
//   [D] elements extend their class's buffer block; blocks beyond the first
//       that a heavy class completes in one tile go straight to their slots;
//   [E] every completed buffer block is written to its slot (one warp per
//       block, coalesced);
//   [F] the remainder of those classes starts their next buffer block.
// A slot is written only after the tile covering it has been read, so the
// stripe is rewritten in place.
//
// Classification uses the branchless tree of Sec. 2 started from a lookup
// table: the splitter range is cut into kCells cells by the leading bits of
// (key - smallest splitter); for each cell the table holds the deepest tree
// node that every key of the cell reaches, so the walk resumes there (the
// start-node table proposed as future work in Sec. 8).  Every step taken is
// a step of the full walk, so the class is exactly the tree's.
#pragma once

#include "level.cuh"

namespace ipsgpu {

constexpr int kCellBits = 12;
constexpr int kCells = 1 << kCellBits;

template <class T>
struct ClsCfg {
    static constexpr bool kSmall = T::D <= 32;
    static constexpr int NT = kSmall ? 1024 : 512;
    // elements per thread and tile: a 48-64 KiB stage for 4..32-byte elements
    static constexpr int EPT =
        T::D == 4 ? 12 : (T::D == 8 ? 8 : (T::D == 16 ? 4 : (T::D == 32 ? 2 : 1)));
    static constexpr int TILE = NT * EPT;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

template <int BYTES>
__device__ __forceinline__ void cp_async(void *dst_smem, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(smem_u32(dst_smem)),
                 "l"(src), "n"(BYTES)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// Tile loader.  The 16-byte aligned interior of the byte range [src, src +
// bytes) goes through one TMA bulk copy issued by thread 0 and completed on
// `bar`; the unaligned head and tail (under 16 bytes each) go through 4-byte
// cp.async copies.  `dst` has the same address modulo 16 as `src`.
__device__ __forceinline__ void tile_load(unsigned char *dst, const unsigned char *src,
                                          uint32_t bytes, uint64_t *bar) {
    const uintptr_t s0 = (uintptr_t)src, s1 = s0 + bytes;
    const uintptr_t lo = (s0 + 15) & ~(uintptr_t)15, hi = s1 & ~(uintptr_t)15;
    const uint32_t tid = threadIdx.x;
    if (tid == 0) {
        if (hi > lo) {
            mbar_arrive_expect_tx(bar, (uint32_t)(hi - lo));
            bulk_load(dst + (lo - s0), reinterpret_cast<const void *>(lo), (uint32_t)(hi - lo), bar);
        } else {
            mbar_arrive_expect_tx(bar, 0);
        }
    }
    // head [s0, min(lo, s1)) and tail [max(hi, lo), s1): at most 3 words each
    if (tid >= 32 && tid < 40) {
        const uint32_t w = tid - 32;
        uintptr_t at;
        if (w < 4)
            at = s0 + 4 * w;
        else
            at = (hi > lo ? hi : lo) + 4 * (w - 4);
        const bool in_head = w < 4 && at < lo && at < s1;
        const bool in_tail = w >= 4 && at < s1 && at >= (hi > lo ? hi : lo);
        if (in_head || in_tail) cp_async<4>(dst + (at - s0), reinterpret_cast<const void *>(at));
    }
    cp_async_commit();
}

// Smallest / largest key whose radix key (T::rkey) equals rk.
template <class T>
__device__ __forceinline__ typename T::K key_lo_of(uint64_t rk) {
    return (typename T::K)rk;
}
template <class T>
__device__ __forceinline__ typename T::K key_hi_of(uint64_t rk) {
    return (typename T::K)rk;
}
// 32-bit keys: cell bounds above the key range clamp to the largest key
template <>
__device__ __forceinline__ uint32_t key_lo_of<TU32>(uint64_t rk) {
    return rk > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)rk;
}
template <>
__device__ __forceinline__ uint32_t key_hi_of<TU32>(uint64_t rk) {
    return rk > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)rk;
}
template <>
__device__ __forceinline__ Key80 key_lo_of<TRec100>(uint64_t rk) {
    Key80 k;
    k.hi = rk;
    k.lo = 0;
    return k;
}
template <>
__device__ __forceinline__ Key80 key_hi_of<TRec100>(uint64_t rk) {
    Key80 k;
    k.hi = rk;
    k.lo = 0xFFFFu;
    return k;
}
template <>
__device__ __forceinline__ Key192 key_lo_of<TQuartet>(uint64_t rk) {
    Key192 k;
    k.a = rk;
    k.b = k.c = 0;
    return k;
}
template <>
__device__ __forceinline__ Key192 key_hi_of<TQuartet>(uint64_t rk) {
    Key192 k;
    k.a = rk;
    k.b = k.c = ~0ull;
    return k;
}
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

// Cell geometry of the start-node table, over x = rk - base (0 below base).
// Linear: cell = min(x >> shift, kCells - 1); with one distinct splitter
// (range 0) every key maps to cell 0, whose entry then is the root.
// Log-scale (for splitters spread over many orders of magnitude): cell =
// 64 e + m, e the position of the leading one of x and m the 6 bits below
// it, so every octave of x gets 64 cells; x = 0 and 1 share cell 0.
constexpr uint32_t kLogMant = 6;
struct CellMap {
    uint64_t base;
    uint32_t shift;
    uint32_t logscale;
    __device__ __forceinline__ uint32_t cell(uint64_t rk) const {
        if (rk < base) return 0;
        const uint64_t x = rk - base;
        if (logscale) {
            if (x < 2) return 0;
            const uint32_t e = 63 - __clzll((long long)x);
            const uint32_t m = e >= kLogMant ? (uint32_t)(x >> (e - kLogMant)) & 63u
                                             : (uint32_t)(x << (kLogMant - e)) & 63u;
            return (e << kLogMant) | m;
        }
        if (shift >= 32) {  // the cell is in the high word
            const uint32_t y = (uint32_t)(x >> 32) >> (shift - 32);
            return y >= (uint32_t)kCells ? (uint32_t)kCells - 1 : y;
        }
        const uint64_t y = x >> shift;
        return y >= (uint64_t)kCells ? (uint32_t)kCells - 1 : (uint32_t)y;
    }
    // rk range [clo, chi] of cell c; false if no rk maps to c
    __device__ bool range(uint32_t c, bool single, uint64_t &clo, uint64_t &chi) const {
        if (!logscale) {
            if (single) {
                clo = 0;
                chi = ~0ull;
                return true;
            }
            clo = c == 0 ? 0 : base + ((uint64_t)c << shift);
            const uint64_t top = base + (((uint64_t)c + 1) << shift) - 1;
            chi = (c == (uint32_t)kCells - 1 || top < base) ? ~0ull : top;
            return c == 0 || clo >= base;  // cells past 2^64 are empty
        }
        const uint32_t e = c >> kLogMant, m = c & 63u;
        uint64_t lo, hi;
        if (c == 0) {
            lo = 0;
            hi = 1;
        } else if (e == 0) {
            return false;
        } else if (e < kLogMant) {
            if (m & ((1u << (kLogMant - e)) - 1)) return false;
            lo = hi = (1ull << e) + (m >> (kLogMant - e));
        } else {
            lo = (64ull + m) << (e - kLogMant);
            hi = lo + (1ull << (e - kLogMant)) - 1;
        }
        const uint64_t room = ~0ull - base;  // largest x
        if (lo > room) return false;
        clo = c == 0 ? 0 : base + lo;
        chi = base + (hi < room ? hi : room);
        return true;
    }
};

// Number of padded splitters s_0 .. s_{K-2} smaller than key x (binary
// search on the sorted splitter array).
template <class T>
__device__ __forceinline__ uint32_t count_less(const typename T::K *spl, uint32_t nleaves,
                                               const typename T::K &x) {
    uint32_t lo = 0, hi = nleaves - 1;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (spl[mid] < x)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// Builds the table.  For a cell with key range [klo, khi], the splitters
// below klo are below every key of the cell and those not below khi are
// below none, so the class index i = #{j : s_j < key} lies in [ja, ja+cnt]
// with ja = #{s_j < klo} and cnt = #{klo <= s_j < khi}.  Entry:
//   cnt <= kMaxCellCmp:  ja | cnt << 9            (i = ja + compares)
//   otherwise:           1 << 31 | depth << 9 | node  (the deepest tree node
//                        every key of the cell reaches; the walk goes on)
// The map (linear or log-scale) is the one that leaves fewer splitter
// intervals in cells that need the walk (judged at each interval's
// midpoint; every interval holds about the same share of the keys).  All
// threads of the CTA call it.
constexpr uint32_t kMaxCellCmp = 3;
template <class T>
__device__ uint32_t cell_entry(const CellMap &cm, uint32_t c, bool single,
                               const typename T::K *tree, const typename T::K *spl,
                               uint32_t nleaves, uint32_t logK) {
    typedef typename T::K K;
    uint64_t clo, chi;
    if (!cm.range(c, single, clo, chi)) return 0x80000000u | 1u;  // unused: walk from the root
    const K klo = key_lo_of<T>(clo), khi = key_hi_of<T>(chi);
    const uint32_t ja = count_less<T>(spl, nleaves, klo);
    const uint32_t jc = count_less<T>(spl, nleaves, khi);
    if (jc - ja <= kMaxCellCmp) return ja | ((jc - ja) << 9);
    uint32_t i = 1, l = 0;
    for (; l < logK; l++) {
        const K a = tree[i];
        if (a < klo)
            i = 2 * i + 1;  // every key of the cell is larger: right
        else if (!(a < khi))
            i = 2 * i;      // no key of the cell is larger: left
        else
            break;
    }
    return 0x80000000u | (l << 9) | i;
}

template <class T>
__device__ void build_start_table(uint32_t *tab, CellMap &cm, const typename T::K *tree,
                                  const typename T::K *spl, uint32_t nleaves, uint32_t logK,
                                  bool tree_only) {
    const uint64_t lo = rk_of_key<T>(spl[0]);
    const uint64_t hi = rk_of_key<T>(spl[nleaves - 1]);
    const uint64_t range = hi - lo;
    const uint32_t nbits = range ? 64 - __clzll((long long)range) : 0;
    const bool single = range == 0;
    CellMap lin, lg;
    lin.base = lg.base = lo;
    lin.shift = nbits > (uint32_t)kCellBits ? nbits - kCellBits : 0;
    lg.shift = 0;
    lin.logscale = 0;
    lg.logscale = 1;
    // which map leaves fewer splitter intervals to the walk
    bool walk_lin = false, walk_lg = false;
    const uint32_t j = threadIdx.x;
    if (!single && j + 1 < nleaves) {
        const uint64_t a = rk_of_key<T>(spl[j]), b = rk_of_key<T>(spl[j + 1]);
        if (b > a) {
            const uint64_t mid = a + (b - a) / 2;
            walk_lin = cell_entry<T>(lin, lin.cell(mid), false, tree, spl, nleaves, logK) >> 31;
            walk_lg = cell_entry<T>(lg, lg.cell(mid), false, tree, spl, nleaves, logK) >> 31;
        }
    }
    const int n_lin = __syncthreads_count(walk_lin);
    const int n_lg = __syncthreads_count(walk_lg);
    cm = (!single && n_lg < n_lin) ? lg : lin;
    // tree_only: every cell starts the walk at the root (Algorithm 1 as printed)
    for (uint32_t c = threadIdx.x; c < (uint32_t)kCells; c += blockDim.x)
        tab[c] = tree_only ? (0x80000000u | 1u)
                           : cell_entry<T>(cm, c, single, tree, spl, nleaves, logK);
}

// Classify EPT keys: the table gives the class index directly or after at
// most kMaxCellCmp comparisons with consecutive splitters; cells holding more
// splitters resume the tree walk (Algorithm 1 style over all elements) from
// their stored node.  Then the equality step of Sec. 2.
template <class T, int EPT>
__device__ __forceinline__ void classify_tab(const typename T::K (&k)[EPT], uint32_t (&c)[EPT],
                                             const typename T::E (&v)[EPT], const uint32_t *tab,
                                             const CellMap &cm, const typename T::K *tree,
                                             const typename T::K *spl, uint32_t logK, bool eq) {
    uint32_t i[EPT], l[EPT];
    bool walk = false;
#pragma unroll
    for (int e = 0; e < EPT; e++) {
        const uint32_t t = tab[cm.cell(T::rkey(v[e]))];
        if (t >> 31) {
            i[e] = t & 511u;
            l[e] = (t >> 9) & 15u;
            walk = true;
        } else {
            const uint32_t ja = t & 511u, cnt = t >> 9;
            uint32_t x = ja;
#pragma unroll
            for (uint32_t q = 0; q < kMaxCellCmp; q++)
                if (q < cnt && spl[ja + q] < k[e]) x++;
            i[e] = x;
            l[e] = 0xFFu;  // resolved
        }
    }
    if (__any_sync(0xffffffffu, walk)) {
        while (true) {
            bool more = false;
#pragma unroll
            for (int e = 0; e < EPT; e++) {
                if (l[e] < logK) {
                    i[e] = 2 * i[e] + (tree[i[e]] < k[e] ? 1u : 0u);
                    l[e]++;
                    more |= l[e] < logK;
                }
            }
            if (!__any_sync(0xffffffffu, more)) break;
        }
#pragma unroll
        for (int e = 0; e < EPT; e++)
            if (l[e] != 0xFFu) i[e] -= 1u << logK;
    }
    if (eq) {
#pragma unroll
        for (int e = 0; e < EPT; e++) c[e] = 2 * i[e] + 1 - (k[e] < spl[i[e]] ? 1u : 0u);
    } else {
#pragma unroll
        for (int e = 0; e < EPT; e++) c[e] = i[e];
    }
}

template <class T>
struct ClsSmem {
    typedef typename T::K K;
    typedef typename T::E E;
    static constexpr int TILE = ClsCfg<T>::TILE;
    static constexpr size_t a16(size_t x) { return (x + 15) & ~(size_t)15; }
    static constexpr size_t o_tree = 0;
    static constexpr size_t o_spl = o_tree + kMaxClasses * sizeof(K);
    static constexpr size_t o_meta = a16(o_spl + kMaxClasses * sizeof(K));
    static constexpr size_t o_cnt = o_meta + kMaxClasses * sizeof(uint2);
    static constexpr size_t o_fill = o_cnt + kMaxClasses * sizeof(uint32_t);
    static constexpr size_t o_tot = o_fill + kMaxClasses * sizeof(uint32_t);
    static constexpr size_t o_tab = o_tot + kMaxClasses * sizeof(uint32_t);
    static constexpr size_t o_stage = a16(o_tab + kCells * sizeof(uint32_t));
    static constexpr size_t o_buf = a16(o_stage + (size_t)TILE * T::D + 16);
    // k buffer blocks of b elements: a level of this sorter has at most k
    // classes (equality buckets included)
    static size_t bytes(uint32_t k, uint32_t b) { return o_buf + (size_t)k * b * T::D; }
};

template <class T>
__global__ void __launch_bounds__(ClsCfg<T>::NT, 1) k_classify(LevelArgs a) {
    typedef typename T::K K;
    typedef typename T::E E;
    typedef ClsSmem<T> L;
    constexpr int NT = ClsCfg<T>::NT;
    constexpr int TILE = ClsCfg<T>::TILE;
    constexpr int EPT = ClsCfg<T>::EPT;
    constexpr int NW = NT / 32;
    extern __shared__ __align__(16) unsigned char smem[];
    K *s_tree = reinterpret_cast<K *>(smem + L::o_tree);
    K *s_spl = reinterpret_cast<K *>(smem + L::o_spl);
    uint2 *meta = reinterpret_cast<uint2 *>(smem + L::o_meta);
    uint32_t *cnt = reinterpret_cast<uint32_t *>(smem + L::o_cnt);
    uint32_t *fill = reinterpret_cast<uint32_t *>(smem + L::o_fill);
    uint32_t *tot = reinterpret_cast<uint32_t *>(smem + L::o_tot);
    uint32_t *tab = reinterpret_cast<uint32_t *>(smem + L::o_tab);
    unsigned char *stage_raw = smem + L::o_stage;
    E *buf = reinterpret_cast<E *>(smem + L::o_buf);
    __shared__ uint32_t sh_wblk;
    __shared__ CellMap sh_cm;
    __shared__ __align__(8) uint64_t sh_bar;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        mbar_init(&sh_bar, 1);
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    }
    uint32_t parity = 0;
    // a balanced wave gives this CTA the stripes of its part; otherwise the
    // stripes are taken round-robin
    const bool parts = a.stripe_first && a.cnt && a.cnt->balanced;
    const uint32_t nstripe = lv_nstripe(a);
    const uint32_t s_begin = parts ? a.stripe_first[blockIdx.x] : blockIdx.x;
    const uint32_t s_end = parts ? a.stripe_first[blockIdx.x + 1] : nstripe;
    const uint32_t s_step = parts ? 1u : gridDim.x;
    for (uint32_t sidx = s_begin; sidx < s_end; sidx += s_step) {
    __syncthreads();
    const StripeDesc sp = a.stripe[sidx];
    const SegDesc sd = a.seg[sp.seg];
    const SegState &st = a.st[sp.seg];
    const uint32_t B = st.B;
    const uint32_t b = sd.b;
    const uint32_t lb = ilog2_floor(b);
    LevelClassifier<T> cl;
    load_classifier<T>(cl, a, sd, st, s_tree, s_spl);
    for (uint32_t j = tid; j < kMaxClasses; j += NT) {
        cnt[j] = 0;
        fill[j] = 0;
        tot[j] = 0;
    }
    if (tid == 0) sh_wblk = 0;
    const E *segbase = reinterpret_cast<const E *>(sd.addr);
    E *segw = reinterpret_cast<E *>(sd.addr);
    const uint64_t e0 = (uint64_t)sp.blk0 * b;
    uint64_t e1 = (uint64_t)(sp.blk0 + sp.nblk) * b;
    if (e1 > sd.n) e1 = sd.n;
    E *out = segw + e0;
    // the stage starts at the stripe's address modulo 16 so that the tile's
    // aligned interior lands on a 16-byte boundary for the bulk copy
    const unsigned char *gsrc = reinterpret_cast<const unsigned char *>(segbase + e0);
    E *stage = reinterpret_cast<E *>(stage_raw + ((uintptr_t)gsrc & 15));
    __syncthreads();
    if (e0 < e1)
        tile_load(reinterpret_cast<unsigned char *>(stage), gsrc,
                  (uint32_t)min((uint64_t)TILE, e1 - e0) * T::D, &sh_bar);
    if (!cl.radix) {
        CellMap cm;
        build_start_table<T>(tab, cm, s_tree, s_spl, st.K, st.logK, a.tree_only != 0);
        if (tid == 0) sh_cm = cm;
    }

    for (uint64_t t0 = e0; t0 < e1; t0 += TILE, parity ^= 1) {
        const uint32_t tcount = (uint32_t)min((uint64_t)TILE, e1 - t0);
        // [A] the tile is in shared memory (bounded wait on the bulk copy)
        const bool landed = mbar_wait_bounded(&sh_bar, parity, a.spin_limit);
        cp_async_wait_all();
        if (__syncthreads_or(!landed)) {
            if (tid == 0) set_status(a.status, IPSGPU_E_TIMEOUT);
            mbar_wait_bounded(&sh_bar, parity, a.spin_limit);
            return;
        }
        // [B] classify and rank
        E v[EPT];
        K k[EPT];
        uint32_t c[EPT], r[EPT];
        uint32_t valid = 0;
#pragma unroll
        for (int e = 0; e < EPT; e++) {
            const uint32_t li = e * NT + tid;
            if (li < tcount) {
                v[e] = stage[li];
                k[e] = T::key(v[e]);
                valid |= 1u << e;
            } else {
                v[e] = stage[0];
                k[e] = T::max_key();
            }
        }
        if (cl.radix) {
#pragma unroll
            for (int e = 0; e < EPT; e++)
                c[e] = (uint32_t)((T::rkey(v[e]) >> cl.shift) & cl.mask);
        } else {
            classify_tab<T, EPT>(k, c, v, tab, sh_cm, s_tree, s_spl, cl.logK, cl.eq);
        }
        // ranks: one shared-memory atomic per element, or one per warp when
        // all its lanes hold the same class (runs of presorted input)
#pragma unroll
        for (int e = 0; e < EPT; e++) {
            const bool ok = (valid >> e) & 1u;
            if (!ok) c[e] = 0xFFFFFFFFu;
            const uint32_t c0 = __shfl_sync(0xffffffffu, c[e], 0);
            r[e] = 0;
            if (__all_sync(0xffffffffu, c[e] == c0) && c0 != 0xFFFFFFFFu) {
                uint32_t base = 0;
                if (lane == 0) base = atomicAdd(&cnt[c0], 32u);
                r[e] = __shfl_sync(0xffffffffu, base, 0) + (uint32_t)lane;
            } else if (ok) {
                r[e] = atomicAdd(&cnt[c[e]], 1u);
            }
        }
        __syncthreads();
        // the stage buffer is free: stream in the next tile
        if (t0 + TILE < e1)
            tile_load(reinterpret_cast<unsigned char *>(stage),
                      reinterpret_cast<const unsigned char *>(segbase + t0 + TILE),
                      (uint32_t)min((uint64_t)TILE, e1 - t0 - TILE) * T::D, &sh_bar);
        // [C] per class: completed blocks and their slots; meta = {old fill
        // | nf << 16 with nf = blocks completed in this tile, first slot}
        // (both halves < 2^16: fill < b and nf <= (b + TILE) / b)
        for (uint32_t j = tid; j < B; j += NT) {
            const uint32_t cc = cnt[j], ff = fill[j];
            const uint32_t nf = (ff + cc) >> lb;
            const uint32_t slot = nf ? atomicAdd(&sh_wblk, nf) : 0u;
            meta[j] = make_uint2(ff | (nf << 16), slot);
            fill[j] = ff + cc - (nf << lb);
            tot[j] += cc;
            cnt[j] = 0;
        }
        __syncthreads();
        // [D] element with in-class position g = fill + rank: g < b extends
        // (and may complete) the class's buffer block; the later blocks a
        // heavy class completes in this tile go straight to their slots; the
        // rest waits until the buffer block has been flushed
        uint32_t gq[EPT];
#pragma unroll
        for (int e = 0; e < EPT; e++) {
            gq[e] = 0xFFFFFFFFu;
            if (c[e] != 0xFFFFFFFFu) {
                const uint2 m = meta[c[e]];
                const uint32_t g = (m.x & 0xFFFFu) + r[e], L = (m.x >> 16) << lb;
                if (g < b)
                    buf[((size_t)c[e] << lb) + g] = v[e];
                else if (g < L)
                    out[((uint64_t)m.y << lb) + g] = v[e];
                else
                    gq[e] = g - L;
            }
        }
        __syncthreads();
        // [E] flush every completed buffer block to its slot (coalesced)
        for (uint32_t j = warp; j < B; j += NW) {
            const uint2 m = meta[j];
            if (m.x >> 16) {
                E *dst = out + ((uint64_t)m.y << lb);
                const E *src = buf + ((size_t)j << lb);
                for (uint32_t o = lane; o < b; o += 32) dst[o] = src[o];
            }
        }
        __syncthreads();
        // [F] the remainder of classes that completed a block
#pragma unroll
        for (int e = 0; e < EPT; e++)
            if (gq[e] != 0xFFFFFFFFu) buf[((size_t)c[e] << lb) + gq[e]] = v[e];
    }
    cp_async_wait_all();
    __syncthreads();
    uint32_t *sc = a.scount + sp.cnt_off;
    for (uint32_t j = tid; j < B; j += NT) sc[j] = tot[j];
    if (tid == 0) a.sfull[sidx] = sh_wblk;
    E *left = reinterpret_cast<E *>(a.arena + sp.left_off);
    for (uint32_t j = warp; j < B; j += NW) {
        const uint32_t f = fill[j];
        for (uint32_t o = lane; o < f; o += 32)
            left[((size_t)j << lb) + o] = buf[((size_t)j << lb) + o];
    }
    }  // stripes
}

}  // namespace ipsgpu

// classify.cuh -- classification with buffer blocks (Sec. 3.1.2 of Axtmann et
// al.), the first half of every partitioning level.
//
// One CTA owns one stripe (a run of whole blocks of its segment).  The stripe
// is read tile by tile; the next tile streams into shared memory by one
// bulk copy (cp.async.bulk, mbarrier) while the current one is processed:
//   [B] every thread classifies its elements and takes its position g in
//       its class's buffer block with a shared-memory atomic on a counter
//       that starts the tile at the block's fill (one atomic per warp when
//       all its lanes share a class);
//   [C] per class, the buffer blocks that fill up in this tile get slots at
//       the front of the stripe (an atomic on the stripe's block counter:
//       the order of full blocks in a stripe is free);
//   [D] elements extend their class's buffer block; blocks beyond the first
//       that a heavy class completes in one tile go straight to their slots;
//   [E] every completed buffer block is written to its slot (a list of
//       flush jobs built in [C]; one warp per block, 16-byte accesses where
//       the stripe's alignment allows);
//   [F] the remainder of those classes starts their next buffer block.
// A slot is written only after the tile covering it has been read, so the
// stripe is rewritten in place.
//
// Classification counts the splitters below the key (the class of Sec. 2's
// branchless tree) through a lookup table addressed by the key's leading
// bits -- the table of start nodes Sec. 8 proposes, in its shortest exact
// form: the splitter range is cut into 2^12 cells; a
// cell's entry holds ja, the number of splitters below every key of the
// cell, and cnt, the number of splitters inside the cell's key range.  The
// class index is ja plus the number of those cnt splitters below the key:
// one compare when the cell holds at most one splitter (nearly every cell
// with k = 256), a binary search over the cell's splitters otherwise.
// IPSGPU_SAMPLESORT_TREE walks every key from the tree's root instead
// (Algorithm 1 as printed, for comparison); both give the same classes.
#pragma once

#include "level.cuh"

namespace ipsgpu {

template <class T>
struct ClsCfg {
    static constexpr bool kSmall = T::D <= 32;
    static constexpr int NT = kSmall ? 1024 : 512;
    // elements per thread and tile: a 48-64 KiB stage for 4..32-byte elements
    static constexpr int EPT =
        T::D == 4 ? 12 : (T::D == 8 ? 8 : (T::D == 16 ? 4 : (T::D == 32 ? 2 : 1)));
    static constexpr int TILE = NT * EPT;
    // cells of the start-node table: 4096 entries of 4 bytes
    static constexpr uint32_t kCellBits = 12;
    static constexpr uint32_t kCells = 1u << kCellBits;
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
// Cell maps of the start-node table.  A key's leading word rk picks a cell:
//   linear:    y = rk >> shift, cell = clamp(y - bc, 0, kCells - 1), with bc
//              = (smallest splitter's rk) >> shift and shift chosen so the
//              splitters span at most kCells cells (kLinHi: shift >= 32, so
//              y comes from the key's high 32-bit word alone)
//   log-scale: x = rk - base (0 below base), cell = 2^mant e + m with e the
//              position of x's leading one and m the mant = cbits - 6 bits
//              below it, so each of the 64 octaves of x gets 2^mant cells
//              (x = 0 and 1: cell 0); for splitters spread over many orders
//              of magnitude
//   single:    one distinct splitter: no table, one compare
enum CellKind : uint32_t { kLinHi = 0, kLinLo = 1, kLog = 2, kSingle = 3 };
struct CellMap {
    uint64_t base;  // log-scale origin (smallest splitter's rk)
    uint64_t bc;    // linear: smallest splitter's rk >> shift
    uint32_t shift;
    uint32_t kind;
    uint32_t cbits;  // log2 of the number of cells
    uint32_t osh;    // linear: a key's offset bits inside its cell, (rk >> osh) & omask
    uint32_t omask;  // (the top min(shift, 22) of the shift bits below the cell index)
    uint32_t pad;
    __device__ __forceinline__ uint32_t top() const { return (1u << cbits) - 1; }
    __device__ __forceinline__ uint32_t offset(uint64_t rk) const {
        return (uint32_t)(rk >> osh) & omask;
    }
    __device__ __forceinline__ uint32_t cell_lin_hi(uint64_t rk) const {
        const uint32_t y = (uint32_t)(rk >> 32) >> (shift - 32);
        const uint32_t b32 = (uint32_t)bc;
        return y <= b32 ? 0u : min(y - b32, top());
    }
    __device__ __forceinline__ uint32_t cell_lin_lo(uint64_t rk) const {
        const uint64_t y = rk >> shift;
        return y <= bc ? 0u : (uint32_t)min(y - bc, (uint64_t)top());
    }
    __device__ __forceinline__ uint32_t cell_log(uint64_t rk) const {
        if (rk < base + 2) return 0;  // also rk < base (x would wrap)
        const uint64_t x = rk - base;
        const uint32_t mant = cbits - 6;
        const uint32_t e = 63 - __clzll((long long)x);
        const uint32_t mm = (1u << mant) - 1;
        const uint32_t m = e >= mant ? (uint32_t)(x >> (e - mant)) & mm
                                     : (uint32_t)(x << (mant - e)) & mm;
        return (e << mant) | m;
    }
    __device__ __forceinline__ uint32_t cell(uint64_t rk) const {
        return kind == kLinHi ? cell_lin_hi(rk) : (kind == kLinLo ? cell_lin_lo(rk) : cell_log(rk));
    }
    // rk range [clo, chi] of cell c; false if no rk maps to c
    __device__ bool range(uint32_t c, uint64_t &clo, uint64_t &chi) const {
        if (kind == kLinHi || kind == kLinLo) {
            const uint64_t ymax = ~0ull >> shift;  // largest y
            if (c > 0 && bc + c > ymax) return false;
            clo = c == 0 ? 0 : (bc + c) << shift;
            chi = (c == top() || bc + c >= ymax) ? ~0ull : ((bc + c + 1) << shift) - 1;
            return true;
        }
        const uint32_t mant = cbits - 6;
        const uint32_t e = c >> mant, m = c & ((1u << mant) - 1);
        uint64_t lo, hi;
        if (c == 0) {
            lo = 0;
            hi = 1;
        } else if (e == 0) {
            return false;
        } else if (e < mant) {
            if (m & ((1u << (mant - e)) - 1)) return false;
            lo = hi = (1ull << e) + (m >> (mant - e));
        } else {
            lo = ((1ull << mant) + m) << (e - mant);
            hi = lo + (1ull << (e - mant)) - 1;
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

// Table entry of a cell with key range [klo, khi] (32 bits).  The splitters
// below klo are below every key of the cell and those not below khi are
// below none, so the class index i = #{j : s_j < key} of a key of the cell
// is ja + #{q < cnt : s_{ja+q} < key}, with ja = #{s_j < klo} and cnt =
// #{klo <= s_j < khi}.  Entry = ja | mode << 8 | x << 10:
//   mode 0: cnt = 0, i = ja
//   mode 1: cnt = 1 and the cell is one step of a linear map, so its keys
//           share every bit above their offset; x = the splitter's offset
//           bits (22 of them): a key with larger offset bits is above it,
//           smaller below; equal offset bits: compare whole keys
//   mode 2: cnt = 1, compare whole keys (cells 0 and last of a linear map,
//           which also take every key beyond the range, and log-scale cells)
//   mode 3: cnt >= 2 (x = cnt): binary search over the cell's splitters
enum : uint32_t { kEntNone = 0, kEntOffset = 1, kEntCompare = 2, kEntSearch = 3 };
template <class T>
__device__ uint32_t cell_entry(const CellMap &cm, uint32_t c, const typename T::K *spl,
                               uint32_t nleaves) {
    uint64_t clo, chi;
    if (!cm.range(c, clo, chi)) return 0;  // no key maps here
    const uint32_t ja = count_less<T>(spl, nleaves, key_lo_of<T>(clo));
    const uint32_t jc = count_less<T>(spl, nleaves, key_hi_of<T>(chi));
    const uint32_t cnt = jc - ja;
    if (cnt == 0) return ja;
    if (cnt >= 2) return ja | (kEntSearch << 8) | (cnt << 10);
    const bool linear = cm.kind == kLinHi || cm.kind == kLinLo;
    if (linear && c != 0 && c != cm.top())
        return ja | (kEntOffset << 8) | (cm.offset(rk_of_key<T>(spl[ja])) << 10);
    return ja | (kEntCompare << 8);
}

// Builds the map and the table.  The map (linear or log-scale) is the one
// that leaves fewer splitter intervals in cells holding two or more
// splitters, whose keys take the slow path (judged at each interval's
// midpoint; every interval holds about the same share of the keys).  All
// threads of the CTA call it.
template <class T>
__device__ void build_start_table(uint32_t *tab, CellMap &cm, const typename T::K *spl,
                                  uint32_t nleaves) {
    constexpr uint32_t kCellBits = ClsCfg<T>::kCellBits;
    constexpr uint32_t kCells = ClsCfg<T>::kCells;
    const uint64_t lo = rk_of_key<T>(spl[0]);
    const uint64_t hi = rk_of_key<T>(spl[nleaves - 1]);
    CellMap lin, lg;
    lin.base = lg.base = lo;
    lin.cbits = lg.cbits = kCellBits;
    lin.pad = lg.pad = 0;
    lg.bc = 0;
    lg.shift = 0;
    lg.kind = kLog;
    lg.osh = 0;
    lg.omask = 0;
    {
        const uint64_t range = hi - lo;
        uint32_t s = range ? 64 - __clzll((long long)range) : 0;
        s = s > kCellBits ? s - kCellBits : 0;
        if (s < 64 && (hi >> s) - (lo >> s) >= (uint64_t)kCells) s++;
        lin.shift = s;
        lin.bc = lo >> s;
        lin.kind = s >= 32 ? kLinHi : kLinLo;
        lin.osh = s > 22 ? s - 22 : 0;
        lin.omask = (1u << (s < 22 ? s : 22)) - 1;
    }
    if (!(spl[0] < spl[nleaves - 1])) {  // one distinct splitter: s_0 < key decides
        cm = lin;
        cm.kind = kSingle;
        return;
    }
    bool slow_lin = false, slow_lg = false;
    const uint32_t j = threadIdx.x;
    if (j + 1 < nleaves - 1) {
        const uint64_t a = rk_of_key<T>(spl[j]), b = rk_of_key<T>(spl[j + 1]);
        if (b > a) {
            const uint64_t mid = a + (b - a) / 2;
            slow_lin = ((cell_entry<T>(lin, lin.cell(mid), spl, nleaves) >> 8) & 3) == kEntSearch;
            slow_lg = ((cell_entry<T>(lg, lg.cell(mid), spl, nleaves) >> 8) & 3) == kEntSearch;
        }
    }
    const int n_lin = __syncthreads_count(slow_lin);
    const int n_lg = __syncthreads_count(slow_lg);
    cm = n_lg < n_lin ? lg : lin;
    for (uint32_t c = threadIdx.x; c < kCells; c += blockDim.x)
        tab[c] = cell_entry<T>(cm, c, spl, nleaves);
}

// Classification kinds of a stripe (uniform over the CTA).
enum ClsKind : uint32_t { kcRadix = 0, kcTable = 1, kcSingle = 2, kcTree = 3 };

// Class indices i = #{s_j < key} of EPT keys whose cells are in i[]: from
// the table entry alone (no splitter in the cell, or the offset bits
// decide); a warp that meets a key needing its splitter finishes it with a
// whole-key compare or, for cells with several splitters, a binary search.
template <class T, int EPT>
__device__ __forceinline__ void resolve_cells(const typename T::K (&k)[EPT], const uint64_t (&rk)[EPT],
                                              uint32_t (&i)[EPT], const uint32_t *tab,
                                              const typename T::K *spl, const CellMap &cm) {
    uint32_t slow = 0;  // bit e: i[e] holds the raw entry
#pragma unroll
    for (int e = 0; e < EPT; e++) {
        const uint32_t t = tab[i[e]];
        const uint32_t mode = (t >> 8) & 3u, x = t >> 10;
        const uint32_t ko = cm.offset(rk[e]);
        const bool hard = mode >= kEntCompare || (mode == kEntOffset && ko == x);
        i[e] = hard ? t : (t & 255u) + ((mode == kEntOffset && ko > x) ? 1u : 0u);
        slow |= hard ? (1u << e) : 0u;
    }
    if (__any_sync(0xffffffffu, slow != 0)) {
#pragma unroll
        for (int e = 0; e < EPT; e++) {
            if (slow & (1u << e)) {
                const uint32_t t = i[e];
                uint32_t lo = t & 255u;
                uint32_t hi = lo + (((t >> 8) & 3u) == kEntSearch ? (t >> 10) : 1u);  // i in [lo, hi]
                while (lo < hi) {
                    const uint32_t mid = (lo + hi) >> 1;  // splitter s_mid below the key?
                    if (spl[mid] < k[e])
                        lo = mid + 1;
                    else
                        hi = mid;
                }
                i[e] = lo;
            }
        }
    }
}

template <class T>
struct ClsSmem {
    typedef typename T::K K;
    typedef typename T::E E;
    static constexpr int TILE = ClsCfg<T>::TILE;
    static constexpr size_t a16(size_t x) { return (x + 15) & ~(size_t)15; }
    static constexpr size_t o_spl = 0;
    static constexpr size_t o_fl = a16(o_spl + kMaxClasses * sizeof(K));
    static constexpr size_t o_sl = o_fl + kMaxClasses * sizeof(uint32_t);
    static constexpr size_t o_cnt = o_sl + kMaxClasses * sizeof(uint32_t);
    static constexpr size_t o_fill = o_cnt + kMaxClasses * sizeof(uint32_t);
    static constexpr size_t o_tot = o_fill + kMaxClasses * sizeof(uint32_t);
    static constexpr size_t o_jobs = o_tot + kMaxClasses * sizeof(uint32_t);
    static constexpr size_t o_tab = o_jobs + kMaxClasses * sizeof(uint2);
    static constexpr size_t o_stage = a16(o_tab + ClsCfg<T>::kCells * sizeof(uint32_t));
    static constexpr size_t o_buf = a16(o_stage + (size_t)TILE * T::D + 16);
    // buffer block c of b elements starts at o_buf + c (b D + 16): the 16
    // bytes of padding spread the blocks over the shared-memory banks
    __host__ __device__ static size_t block_pitch(uint32_t b) { return (size_t)b * T::D + 16; }
    // k buffer blocks: a level of this sorter has at most k classes
    // (equality buckets included)
    static size_t bytes(uint32_t k, uint32_t b) { return o_buf + (size_t)k * block_pitch(b); }
};

// Copies one block of BB bytes (a multiple of 16) from shared memory to
// global memory with one warp, in u-byte units (16, 8 or 4: what the
// global address allows; shared memory is 16-byte aligned).
__device__ __forceinline__ void warp_flush_block(unsigned char *dst, const unsigned char *src,
                                                 uint32_t BB, int lane, int u) {
    if (u == 16) {
        for (uint32_t o = (uint32_t)lane * 16; o < BB; o += 512)
            *reinterpret_cast<uint4 *>(dst + o) = *reinterpret_cast<const uint4 *>(src + o);
    } else if (u == 8) {
        for (uint32_t o = (uint32_t)lane * 8; o < BB; o += 256)
            *reinterpret_cast<uint2 *>(dst + o) = *reinterpret_cast<const uint2 *>(src + o);
    } else {
        for (uint32_t o = (uint32_t)lane * 4; o < BB; o += 128)
            *reinterpret_cast<uint32_t *>(dst + o) = *reinterpret_cast<const uint32_t *>(src + o);
    }
}

template <class T>
__global__ void __launch_bounds__(ClsCfg<T>::NT, 1) k_classify(LevelArgs a) {
    typedef typename T::K K;
    typedef typename T::E E;
    typedef ClsSmem<T> L;
    constexpr int NT = ClsCfg<T>::NT;
    constexpr int TILE = ClsCfg<T>::TILE;
    constexpr int EPT = ClsCfg<T>::EPT;
    constexpr int NW = NT / 32;
    static_assert(kMaxClasses <= NT, "[C] gives every class its own thread");
    extern __shared__ __align__(16) unsigned char smem[];
    K *s_spl = reinterpret_cast<K *>(smem + L::o_spl);
    uint32_t *fl = reinterpret_cast<uint32_t *>(smem + L::o_fl);
    uint32_t *sl = reinterpret_cast<uint32_t *>(smem + L::o_sl);
    uint32_t *cnt = reinterpret_cast<uint32_t *>(smem + L::o_cnt);
    uint32_t *fill = reinterpret_cast<uint32_t *>(smem + L::o_fill);
    uint32_t *tot = reinterpret_cast<uint32_t *>(smem + L::o_tot);
    uint2 *jobs = reinterpret_cast<uint2 *>(smem + L::o_jobs);
    uint32_t *tab = reinterpret_cast<uint32_t *>(smem + L::o_tab);
    unsigned char *stage_raw = smem + L::o_stage;
    unsigned char *bufr = smem + L::o_buf;
    __shared__ uint32_t sh_wblk, sh_njobs;
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
    const uint32_t BB = b * T::D;
    const uint32_t pitch = (uint32_t)L::block_pitch(b);
    // the tree (Algorithm 1's walk) is read from global memory: it is only
    // walked by IPSGPU_SAMPLESORT_TREE, which exists for comparison
    LevelClassifier<T> cl;
    load_classifier<T>(cl, a, sd, st, nullptr, s_spl);
    const K *g_tree = seg_tree<T>(a, sd);
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
    // widest unit both a block of the stripe and shared memory allow
    const int fu = access_unit((uint64_t)(uintptr_t)out);
    // the stage starts at the stripe's address modulo 16 so that the tile's
    // aligned interior lands on a 16-byte boundary for the bulk copy
    const unsigned char *gsrc = reinterpret_cast<const unsigned char *>(segbase + e0);
    E *stage = reinterpret_cast<E *>(stage_raw + ((uintptr_t)gsrc & 15));
    __syncthreads();
    if (e0 < e1)
        tile_load(reinterpret_cast<unsigned char *>(stage), gsrc,
                  (uint32_t)min((uint64_t)TILE, e1 - e0) * T::D, &sh_bar);
    uint32_t kind = kcRadix;
    if (!cl.radix) {
        if (a.tree_only) {
            kind = kcTree;
        } else {
            CellMap cm;
            build_start_table<T>(tab, cm, s_spl, st.K);
            if (tid == 0) sh_cm = cm;
            kind = cm.kind == kSingle ? kcSingle : kcTable;
        }
    }

    for (uint64_t t0 = e0; t0 < e1; t0 += TILE, parity ^= 1) {
        const uint32_t tcount = (uint32_t)min((uint64_t)TILE, e1 - t0);
        // [A] the tile is in shared memory (bounded wait on the bulk copy)
        const bool landed = mbar_wait_bounded(&sh_bar, parity, a.spin_limit);
        cp_async_wait_all();
        if (tid == 0) sh_njobs = 0;
        if (__syncthreads_or(!landed)) {
            if (tid == 0) set_status(a.status, IPSGPU_E_TIMEOUT);
            mbar_wait_bounded(&sh_bar, parity, a.spin_limit);
            return;
        }
        // [B] classify and rank; elements past the tile's end get class ~0
        E v[EPT];
        K k[EPT];
        uint32_t c[EPT], r[EPT];
        const bool full = tcount == (uint32_t)TILE;
#pragma unroll
        for (int e = 0; e < EPT; e++) {
            const uint32_t li = e * NT + tid;
            v[e] = stage[full || li < tcount ? li : 0];
            k[e] = T::key(v[e]);
        }
        if (kind == kcRadix) {
#pragma unroll
            for (int e = 0; e < EPT; e++)
                c[e] = (uint32_t)((T::rkey(v[e]) >> cl.shift) & cl.mask);
        } else {
            if (kind == kcTable) {
                const CellMap cm = sh_cm;
                uint64_t rk[EPT];
#pragma unroll
                for (int e = 0; e < EPT; e++) rk[e] = T::rkey(v[e]);
                if (cm.kind == kLinHi) {
#pragma unroll
                    for (int e = 0; e < EPT; e++) c[e] = cm.cell_lin_hi(rk[e]);
                } else if (cm.kind == kLinLo) {
#pragma unroll
                    for (int e = 0; e < EPT; e++) c[e] = cm.cell_lin_lo(rk[e]);
                } else {
#pragma unroll
                    for (int e = 0; e < EPT; e++) c[e] = cm.cell_log(rk[e]);
                }
                resolve_cells<T, EPT>(k, rk, c, tab, s_spl, cm);
            } else if (kind == kcSingle) {
                // one distinct splitter s: keys <= s have index 0, the rest K - 1
#pragma unroll
                for (int e = 0; e < EPT; e++) c[e] = s_spl[0] < k[e] ? st.K - 1 : 0u;
            } else {
                // Algorithm 1 as printed: every key walks the tree from the root
#pragma unroll
                for (int e = 0; e < EPT; e++) {
                    uint32_t x = 1;
                    for (uint32_t l = 0; l < cl.logK; l++) x = 2 * x + (g_tree[x] < k[e] ? 1u : 0u);
                    c[e] = x - st.K;
                }
            }
            if (cl.eq) {
#pragma unroll
                for (int e = 0; e < EPT; e++) c[e] = 2 * c[e] + 1 - (k[e] < s_spl[c[e]] ? 1u : 0u);
            }
        }
        if (!full) {
#pragma unroll
            for (int e = 0; e < EPT; e++)
                if ((uint32_t)(e * NT + tid) >= tcount) c[e] = 0xFFFFFFFFu;
        }
        // ranks: one shared-memory atomic per element, or one per warp when
        // all its elements share a class (runs of presorted input)
        {
            const uint32_t c0 = __shfl_sync(0xffffffffu, c[0], 0);
            bool same = c0 != 0xFFFFFFFFu;
#pragma unroll
            for (int e = 0; e < EPT; e++) same = same && c[e] == c0;
            if (__all_sync(0xffffffffu, same)) {
                uint32_t base = 0;
                if (lane == 0) base = atomicAdd(&cnt[c0], 32u * EPT);
                base = __shfl_sync(0xffffffffu, base, 0);
#pragma unroll
                for (int e = 0; e < EPT; e++) r[e] = base + (uint32_t)(e * 32 + lane);
            } else {
#pragma unroll
                for (int e = 0; e < EPT; e++)
                    r[e] = c[e] != 0xFFFFFFFFu ? atomicAdd(&cnt[c[e]], 1u) : 0u;
            }
        }
        __syncthreads();
        // the stage buffer is free: stream in the next tile
        if (t0 + TILE < e1)
            tile_load(reinterpret_cast<unsigned char *>(stage),
                      reinterpret_cast<const unsigned char *>(segbase + t0 + TILE),
                      (uint32_t)min((uint64_t)TILE, e1 - t0 - TILE) * T::D, &sh_bar);
        // [C] per class (cnt = fill before the tile + the tile's elements):
        // blocks completed in this tile and their slots at the front of the
        // stripe; fl = elements that go to completed blocks (nf b), sl =
        // first slot; the class's buffer block, if completed, is a flush
        // job; cnt restarts at the new fill.  B <= 256 <= NT: thread j takes
        // class j; slots and job entries are handed out one atomic per warp
        if ((uint32_t)(tid & ~31) < B) {
            const uint32_t j = tid;
            const bool act = j < B;
            const uint32_t ct = act ? cnt[j] : 0u, ff = act ? fill[j] : 0u;
            const uint32_t cc = ct - ff;
            const uint32_t nf = ct >> lb;
            uint32_t x = nf;  // inclusive warp scan of nf
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            const uint32_t jb = __ballot_sync(0xffffffffu, nf != 0);
            uint32_t s0 = 0, q0 = 0;
            if (lane == 31 && x) {
                s0 = atomicAdd(&sh_wblk, x);
                q0 = atomicAdd(&sh_njobs, (uint32_t)__popc(jb));
            }
            s0 = __shfl_sync(0xffffffffu, s0, 31);
            q0 = __shfl_sync(0xffffffffu, q0, 31);
            const uint32_t slot = s0 + x - nf;
            if (nf) jobs[q0 + __popc(jb & ((1u << lane) - 1))] = make_uint2(j, slot);
            if (act) {
                fl[j] = nf << lb;
                sl[j] = slot;
                fill[j] = ct & (b - 1);
                tot[j] += cc;
                cnt[j] = ct & (b - 1);
            }
        }
        __syncthreads();
        // [D] element with in-class position g: g < b extends (and may
        // complete) the class's buffer block; the later blocks a heavy class
        // completes in this tile go straight to their slots; the rest waits
        // until the buffer block has been flushed
        uint32_t gq[EPT];
#pragma unroll
        for (int e = 0; e < EPT; e++) {
            gq[e] = 0xFFFFFFFFu;
            if (c[e] != 0xFFFFFFFFu) {
                const uint32_t g = r[e];
                if (g < b) {
                    reinterpret_cast<E *>(bufr + c[e] * pitch)[g] = v[e];
                } else {
                    const uint32_t Lq = fl[c[e]];
                    if (g < Lq)
                        out[((uint64_t)sl[c[e]] << lb) + g] = v[e];
                    else
                        gq[e] = g - Lq;
                }
            }
        }
        __syncthreads();
        // [E] flush every completed buffer block to its slot (one warp each)
        const uint32_t nj = sh_njobs;
        for (uint32_t q = warp; q < nj; q += NW) {
            const uint2 jb = jobs[q];
            warp_flush_block(reinterpret_cast<unsigned char *>(out + ((uint64_t)jb.y << lb)),
                             bufr + jb.x * pitch, BB, lane, fu);
        }
        __syncthreads();
        // [F] the remainder of classes that completed a block
#pragma unroll
        for (int e = 0; e < EPT; e++)
            if (gq[e] != 0xFFFFFFFFu) reinterpret_cast<E *>(bufr + c[e] * pitch)[gq[e]] = v[e];
    }
    cp_async_wait_all();
    __syncthreads();
    uint32_t *sc = a.scount + sp.cnt_off;
    for (uint32_t j = tid; j < B; j += NT) sc[j] = tot[j];
    if (tid == 0) a.sfull[sidx] = sh_wblk;
    E *left = reinterpret_cast<E *>(a.arena + sp.left_off);
    for (uint32_t j = warp; j < B; j += NW) {
        const uint32_t f = fill[j];
        const E *src = reinterpret_cast<const E *>(bufr + j * pitch);
        for (uint32_t o = lane; o < f; o += 32) left[((size_t)j << lb) + o] = src[o];
    }
    }  // stripes
}

}  // namespace ipsgpu

// graph.cuh -- the segmented batch run entirely on the device: the recursion
// of Sec. 3.2 planned level by level by kernels instead of the host, so the
// whole batch is one fixed sequence of launches (capturable in a CUDA graph).
//
//   k_g_init          splits the input arrays (offsets into one array, a list
//                     of (address, length) pairs, or one whole array): one
//                     element or fewer: done; at most the base-case size:
//                     base list; else level 0
//   k_g_plan          one CTA plans a level: class budget, stripes, CTAs and
//                     arena offsets of every segment (prefix sums)
//   k_g_fill_stripes  stripe descriptors and the CTA -> segment map
//   level kernels     as for a host-planned level, counts read from memory
//   k_g_emit          children of every bucket: done (equality bucket, at
//                     most one element, radix digits exhausted), base list,
//                     or the next level's list
#pragma once

#include "common.cuh"

namespace ipsgpu {

constexpr int kPlanThreads = 1024;
constexpr uint32_t kMinStripeElems = 1u << 15;

struct GList {
    uint64_t addr, n;          // device byte address of the first element, elements
    uint32_t shift, pad;
};

struct GraphArgs {
    LevelArgs lv;              // the level's arrays (counts come from `counts`)
    LevelCounts *counts;       // device: counts of the level being run
    GList *list[2];            // ping-pong lists of segments to partition
    uint32_t *list_count[2];
    uint64_t *base_list;       // (address, n) pairs for the base case
    uint32_t *base_count;
    uint32_t *invalid;         // set when an input segment had bad offsets
    // input, one of: offsets (nseg_in + 1 element offsets into lv.data),
    // segs (nseg_in (address, n) pairs), or neither (all of lv.data)
    const uint64_t *offsets;
    const uint64_t *segs;
    const int *skip_flags;     // if set: skip the input when flags[0] or flags[1]
    uint64_t nseg_in;
    uint64_t n_total;          // elements of lv.data (offsets mode, single array)
    uint32_t elem_bytes, elem_align;
    uint32_t list_cap, base_cap, seg_cap, stripe_cap, cta_cap, cls_cap, cnt_cap;
    uint32_t smax, k, b, nsm, kbits, keybits;
    uint64_t arena_bytes, sarr_bytes, keys_bytes;
    int algo;                  // 0 samplesort, 1 radix
    int levels;
};

__device__ inline uint32_t g_next_pow2(uint64_t x) {
    uint32_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

// class budget of a segment: the adaptive k of Sec. 3.2, aimed at children
// of about half the base-case size (same rule as the host planner)
__device__ inline uint32_t g_class_budget(const GraphArgs &g, uint64_t n) {
    const uint64_t half = g.smax / 2;
    uint64_t want = g_next_pow2((n + half - 1) / half);
    if (want < 4) want = 4;
    if (want > g.k) want = g.k;
    return (uint32_t)want;
}

__device__ inline uint64_t g_al256(uint64_t x) { return (x + 255) & ~(uint64_t)255; }

// Appends to a bounded list.  An append past the capacity is undone, so once
// the appending kernel has finished the count never exceeds the capacity and
// every entry below it is written; the overflow is reported as E_NOMEM.
__device__ inline void g_push_base(const GraphArgs &g, uint64_t addr, uint64_t n) {
    const uint32_t q = atomicAdd(g.base_count, 1u);
    if (q < g.base_cap) {
        g.base_list[2 * q] = addr;
        g.base_list[2 * q + 1] = n;
    } else {
        atomicSub(g.base_count, 1u);
        set_status(g.lv.status, IPSGPU_E_NOMEM);
    }
}
__device__ inline void g_push_list(const GraphArgs &g, int which, const GList &e) {
    const uint32_t q = atomicAdd(g.list_count[which], 1u);
    if (q < g.list_cap) {
        g.list[which][q] = e;
    } else {
        atomicSub(g.list_count[which], 1u);
        set_status(g.lv.status, IPSGPU_E_NOMEM);
    }
}

// Arena bytes of a segment: cleanup staging (C blocks) directly followed by
// the overflow block, then C leftover buffer blocks per stripe.
template <class T>
__device__ inline uint64_t g_stage_bytes(uint32_t C, uint32_t b) {
    return g_al256((uint64_t)C * b * T::D + (uint64_t)b * T::D);
}
template <class T>
__device__ inline uint64_t g_left_bytes(uint32_t C, uint32_t b) {
    return g_al256((uint64_t)C * b * T::D);
}

// Input segments [i0, i1).  Offsets must be non-decreasing and within the
// data array, listed arrays aligned to the element type; a segment that is
// not is skipped, and k_g_finish reports E_INVAL once the valid segments are
// sorted.  Segments of at most the base-case size go to the base list, the
// others to the first level.
static __global__ void __launch_bounds__(256) k_g_init(GraphArgs g, uint64_t i0, uint64_t i1) {
    if (g.skip_flags && (g.skip_flags[0] || g.skip_flags[1])) return;  // sorted (or reversed)
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = i0 + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < i1; i += stride) {
        uint64_t addr, n;
        if (g.offsets) {
            const uint64_t b0 = g.offsets[i], b1 = g.offsets[i + 1];
            if (b1 < b0 || b1 > g.n_total) {
                *g.invalid = 1;
                continue;
            }
            addr = (uint64_t)(uintptr_t)g.lv.data + b0 * g.elem_bytes;
            n = b1 - b0;
        } else if (g.segs) {
            addr = g.segs[2 * i];
            n = g.segs[2 * i + 1];
            if ((n > 0 && (addr == 0 || addr % g.elem_align)) || n > (1ull << 40)) {
                *g.invalid = 1;
                continue;
            }
        } else {
            addr = (uint64_t)(uintptr_t)g.lv.data;
            n = g.n_total;
        }
        if (n <= 1) continue;
        if (n <= g.smax)
            g_push_base(g, addr, n);
        else
            g_push_list(g, 0, GList{addr, n, g.keybits > g.kbits ? g.keybits - g.kbits : 0u, 0u});
    }
}

// Per-segment plan quantities.
struct GPlanItem {
    uint32_t C, p, nc;
    uint64_t arena, sarr, keys, cnt;
};

template <class T>
__device__ inline GPlanItem g_item(const GraphArgs &g, uint64_t n, uint64_t stripe_elems,
                                   uint64_t bpc) {
    GPlanItem it;
    it.C = g.algo == 1 ? (1u << g.kbits) : g_class_budget(g, n);
    const uint64_t nb = (n + g.b - 1) / g.b;
    uint64_t p = (n + stripe_elems - 1) / stripe_elems;
    if (p < 1) p = 1;
    if (p > nb) p = nb;
    uint64_t nc = (nb + bpc - 1) / bpc;
    if (nc < 1) nc = 1;
    it.p = (uint32_t)p;
    it.nc = (uint32_t)nc;
    it.arena = g_stage_bytes<T>(it.C, g.b) + p * g_left_bytes<T>(it.C, g.b);
    it.sarr = seg_arrays_bytes(it.C);
    it.keys = ((uint64_t)2 * it.C * sizeof(typename T::K) + 15) & ~(uint64_t)15;
    it.cnt = (uint64_t)it.C * p;
    return it;
}

template <class T>
__global__ void __launch_bounds__(kPlanThreads) k_g_plan(GraphArgs g, int L) {
    constexpr int NV = 7;  // stripes, ctas, classes, arena, sarr, keys, counts
    __shared__ unsigned long long red[2][32];
    __shared__ unsigned long long wsum[NV][32];
    __shared__ int sh_bad;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const GList *in = g.list[L & 1];
    uint32_t nin = *g.list_count[L & 1];
    if (tid == 0) {
        *g.list_count[(L + 1) & 1] = 0;
        *g.base_count = 0;  // the previous base-case launch has consumed it
        sh_bad = 0;
    }
    if (nin > g.list_cap) nin = g.list_cap;
    if (nin > g.seg_cap) {
        if (tid == 0) set_status(g.lv.status, IPSGPU_E_NOMEM);
        nin = 0;
    }
    // pass 1: elements and blocks of the level
    unsigned long long te = 0, tb = 0;
    for (uint32_t i = tid; i < nin; i += kPlanThreads) {
        te += in[i].n;
        tb += (in[i].n + g.b - 1) / g.b;
    }
    for (int o = 16; o > 0; o >>= 1) {
        te += __shfl_xor_sync(0xffffffffu, te, o);
        tb += __shfl_xor_sync(0xffffffffu, tb, o);
    }
    if (lane == 0) {
        red[0][warp] = te;
        red[1][warp] = tb;
    }
    __syncthreads();
    te = 0;
    tb = 0;
    for (int w = 0; w < kPlanThreads / 32; w++) {
        te += red[0][w];
        tb += red[1][w];
    }
    uint64_t stripe_elems = te / (2 * (uint64_t)g.nsm);
    if (stripe_elems < kMinStripeElems) stripe_elems = kMinStripeElems;
    stripe_elems = (stripe_elems + g.b - 1) / g.b * g.b;
    uint64_t bpc = tb / (8 * (uint64_t)g.nsm);
    if (bpc < 32) bpc = 32;
    // pass 2: each thread owns a contiguous range of segments
    const uint32_t per = (nin + kPlanThreads - 1) / kPlanThreads;
    const uint32_t r0 = min(nin, tid * per), r1 = min(nin, r0 + per);
    unsigned long long loc[NV] = {0, 0, 0, 0, 0, 0, 0};
    for (uint32_t i = r0; i < r1; i++) {
        const GPlanItem it = g_item<T>(g, in[i].n, stripe_elems, bpc);
        loc[0] += it.p;
        loc[1] += it.nc;
        loc[2] += it.C;
        loc[3] += it.arena;
        loc[4] += it.sarr;
        loc[5] += it.keys;
        loc[6] += it.cnt;
    }
    // exclusive scan of the seven sums over threads
    unsigned long long incl[NV], excl[NV], tot[NV];
#pragma unroll
    for (int v = 0; v < NV; v++) {
        unsigned long long x = loc[v];
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        incl[v] = x;
        if (lane == 31) wsum[v][warp] = x;
    }
    __syncthreads();
#pragma unroll
    for (int v = 0; v < NV; v++) {
        unsigned long long before = 0, all = 0;
        for (int w = 0; w < kPlanThreads / 32; w++) {
            if (w < warp) before += wsum[v][w];
            all += wsum[v][w];
        }
        excl[v] = before + incl[v] - loc[v];
        tot[v] = all;
    }
    if (tid == 0 &&
        (tot[0] > g.stripe_cap || tot[1] > g.cta_cap || tot[2] > g.cls_cap || tot[3] > g.arena_bytes ||
         tot[4] > g.sarr_bytes || tot[5] > g.keys_bytes || tot[6] > g.cnt_cap ||
         2 * (tot[0] + tot[2]) + 4 * (uint64_t)nin > g.lv.move_cap)) {
        set_status(g.lv.status, IPSGPU_E_NOMEM);
        sh_bad = 1;
    }
    __syncthreads();
    if (sh_bad) nin = 0;
    // pass 3: descriptors with running offsets
    for (uint32_t i = r0; i < r1 && nin; i++) {
        const GPlanItem it = g_item<T>(g, in[i].n, stripe_elems, bpc);
        SegDesc d;
        d.addr = in[i].addr;
        d.n = in[i].n;
        d.b = g.b;
        d.C = it.C;
        d.stripe0 = (uint32_t)excl[0];
        d.nstripes = it.p;
        d.cta0 = (uint32_t)excl[1];
        d.ncta = it.nc;
        d.cls0 = (uint32_t)excl[2];
        d.stage_off = excl[3];
        d.arr_off = excl[4];
        d.key_off = excl[5];
        d.cnt0 = (uint32_t)excl[6];
        d.mode = g.algo == 1 ? 2u : 0u;
        d.radix_shift = in[i].shift;
        d.radix_bits = g.kbits;
        d.nsplit = 0;
        d.eq_given = 0;
        const_cast<SegDesc *>(g.lv.seg)[i] = d;
        excl[0] += it.p;
        excl[1] += it.nc;
        excl[2] += it.C;
        excl[3] += it.arena;
        excl[4] += it.sarr;
        excl[5] += it.keys;
        excl[6] += it.cnt;
    }
    if (tid == 0) {
        LevelCounts c;
        c.nseg = nin;
        c.nstripe = nin ? (uint32_t)tot[0] : 0u;
        c.ncta = nin ? (uint32_t)tot[1] : 0u;
        c.ncls = nin ? (uint32_t)tot[2] : 0u;
        *g.counts = c;
    }
}

// Stripe descriptors and the CTA -> segment map of the planned level.
template <class T>
__global__ void __launch_bounds__(256) k_g_fill_stripes(GraphArgs g) {
    const LevelCounts c = *g.counts;
    const uint32_t stride = gridDim.x * blockDim.x;
    const uint32_t t0 = blockIdx.x * blockDim.x + threadIdx.x;
    for (uint32_t i = t0; i < c.nstripe; i += stride) {
        uint32_t lo = 0, hi = c.nseg;  // last segment with stripe0 <= i
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (g.lv.seg[mid].stripe0 <= i)
                lo = mid;
            else
                hi = mid;
        }
        const SegDesc sd = g.lv.seg[lo];
        const uint64_t nb = (sd.n + sd.b - 1) / sd.b;
        const uint32_t q = i - sd.stripe0, p = sd.nstripes;
        StripeDesc s;
        s.seg = lo;
        s.blk0 = (uint32_t)(q * nb / p);
        s.nblk = (uint32_t)((q + 1) * nb / p - q * nb / p);
        s.cnt_off = sd.cnt0 + q * sd.C;
        s.left_off = sd.stage_off + g_stage_bytes<T>(sd.C, sd.b) +
                     (uint64_t)q * g_left_bytes<T>(sd.C, sd.b);
        const_cast<StripeDesc *>(g.lv.stripe)[i] = s;
    }
    uint32_t *cta_seg = const_cast<uint32_t *>(g.lv.cta_seg);
    for (uint32_t i = t0; i < c.ncta; i += stride) {
        uint32_t lo = 0, hi = c.nseg;  // last segment with cta0 <= i
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (g.lv.seg[mid].cta0 <= i)
                lo = mid;
            else
                hi = mid;
        }
        cta_seg[i] = lo;
    }
}

// Children of every (segment, class) of level L.
template <class T>
__global__ void __launch_bounds__(256) k_g_emit(GraphArgs g, int L) {
    if (*(volatile int *)g.lv.status != 0) return;  // an error: leave the data as is
    const LevelCounts c = *g.counts;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < c.ncls; q += stride) {
        uint32_t lo = 0, hi = c.nseg;  // last segment with cls0 <= q
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (g.lv.seg[mid].cls0 <= q)
                lo = mid;
            else
                hi = mid;
        }
        const SegDesc sd = g.lv.seg[lo];
        const SegState st = g.lv.st[lo];
        const uint32_t j = q - sd.cls0;
        if (j >= st.B) continue;
        if (st.eq && (j & 1) && j + 1 < st.B) continue;  // equality bucket: one key
        const SegArrays ar = seg_arrays(g.lv.sarr, sd);
        const uint64_t b0 = ar.bb[j], b1 = ar.bb[j + 1];
        if (b1 <= b0 + 1) continue;
        const uint64_t n = b1 - b0;
        uint32_t shift = 0;
        if (g.algo == 1) {
            if (sd.radix_shift == 0) continue;  // every key bit used: equal keys
            shift = sd.radix_shift >= g.kbits ? sd.radix_shift - g.kbits : 0u;
        }
        if (n <= g.smax) {
            g_push_base(g, sd.addr + b0 * T::D, n);
        } else if (L + 1 < g.levels) {
            g_push_list(g, (L + 1) & 1, GList{sd.addr + b0 * T::D, n, shift, 0u});
        } else {
            set_status(g.lv.status, IPSGPU_E_INTERNAL);  // deeper than planned
        }
    }
}

// Last launch of a batch: bad input offsets become E_INVAL in the status word
// (unless an earlier error is already recorded) and the flag is cleared.
static __global__ void k_g_finish(GraphArgs g) {
    if (threadIdx.x == 0 && blockIdx.x == 0 && *g.invalid) {
        set_status(g.lv.status, IPSGPU_E_INVAL);
        *g.invalid = 0;
    }
}

}  // namespace ipsgpu

// graph.cuh -- the recursion of Sec. 3.2 run entirely on the device.
//
// Segments that still need a partitioning step wait in a FIFO ring.  The
// work proceeds in waves; one wave is
//   k_g_feed          takes the next input arrays: one element or fewer:
//                     done; at most the base-case size: base list; else ring
//   k_g_plan          one CTA takes the longest prefix of the ring whose
//                     class budgets, stripes, CTAs and arena bytes fit the
//                     sorter's fixed capacities, and lays it out
//   k_g_fill_stripes  stripe descriptors and the CTA -> segment map
//   level kernels     one partitioning step of every taken segment (level.cuh,
//                     classify.cuh; work counts read from memory)
//   k_g_emit          children of every bucket: done (equality bucket, at
//                     most one element, radix digits exhausted), base list,
//                     or the ring's tail
//   k_base            the base case of the wave's base list
//   k_g_advance       consumes the taken prefix and the fed inputs and
//                     decides whether another wave follows
// so scratch is bounded by the capacities, not by n, however many segments
// a level has (the paper bounds it by the number of threads in the same
// way).  The waves run inside a conditional WHILE node of one CUDA graph
// (k_g_advance sets its condition), or, when per-kernel timing is on, from a
// host loop that reads the same decision back.
#pragma once

#include "common.cuh"

namespace ipsgpu {

constexpr int kPlanThreads = 1024;
constexpr uint32_t kMinStripeElems = 1u << 15;

struct GList {
    uint64_t addr, n;  // device byte address of the first element, elements
    uint64_t rlo, rhi; // bounds of the elements' leading key word (rlo > rhi: not known)
    uint32_t shift;    // radix: next digit is key bits [shift, shift + kbits)
    uint32_t pad;
};

// Bounds of every T::rkey in a child of a partitioned segment, from the
// parent's bounds and the class's splitters (class i of the tree holds keys
// s_{i-1} < key <= s_i; with equality buckets class 2i holds s_{i-1} < key <
// s_i and class 2K - 1 keys above every splitter) or from its radix digit.
// Loose bounds stay correct (every key lies inside), an unknown parent
// bound on an edge class becomes the type's whole range.
struct RBounds {
    uint64_t lo, hi;
};

// What one run sorts; written by k_g_job before the run.
struct GJob {
    unsigned char *data;      // offsets mode and single-array mode
    const uint64_t *offsets;  // nseg_in + 1 element offsets into data, or null
    const uint64_t *segs;     // nseg_in (address, n) pairs, or null
    const int *skip_flags;    // if non-null and flags[0] or flags[1]: skip the input
    const unsigned long long *radix_mm;  // single array, radix: key min and max (or null)
    uint64_t nseg_in;         // input arrays (1 in single-array mode)
    uint64_t n_total;         // elements of data (offsets and single-array mode)
    uint32_t max_waves;
    uint32_t pad;
};

// Progress of a run, in device memory.
struct GState {
    LevelCounts counts;  // work counts of the wave's partitioning step
    uint64_t in_head;    // input arrays consumed
    uint64_t head, tail; // ring counters (entry i lives at ring[i % ring_cap])
    uint32_t feed;       // input arrays the current wave feeds
    uint32_t take;       // ring entries the current wave partitions
    uint32_t base_count; // base list entries of the current wave
    uint32_t wave;
    uint32_t invalid;    // an input array had bad offsets or a bad address
    uint32_t more;       // decision of the last k_g_advance
    uint64_t elems;      // elements partitioned by the current wave
    uint64_t base_elems; // elements of the current wave's base list
    uint64_t last_elems, last_base_elems;  // the same of the wave that ended last
    uint64_t part_q, part_blocks;  // balanced waves: blocks per part, blocks taken
};

// Fixed for a sorter: its scratch and capacities.
struct GraphArgs {
    LevelArgs lv;       // arrays of a partitioning step (lv.cnt -> state->counts)
    GJob *job;
    GState *state;
    GList *ring;
    uint64_t *base_list;  // (address, n) pairs for the base case
    uint32_t *stripe_first;  // nparts + 1 entries
    uint32_t nparts;         // classification CTAs of a wave (one per SM)
    uint32_t pad2;
    uint32_t ring_cap, base_cap, feed_cap, seg_cap, stripe_cap, cta_cap, cls_cap, cnt_cap;
    uint32_t smax, k, b, nsm, kbits, keybits, elem_bytes, elem_align;
    uint32_t perm_ctas;      // permutation CTAs resident at once (the wave's grid)
    uint64_t arena_bytes, sarr_bytes, keys_bytes;
    int algo;  // 0 samplesort, 1 radix
    int pad;
};

__device__ inline uint32_t g_next_pow2(uint64_t x) {
    uint32_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

// class budget of a segment: the adaptive k of Sec. 3.2, aimed at children
// of about half the base-case size
__device__ inline uint32_t g_class_budget(const GraphArgs &g, uint64_t n) {
    const uint64_t half = g.smax / 2;
    uint64_t want = g_next_pow2((n + half - 1) / half);
    if (want < 4) want = 4;
    if (want > g.k) want = g.k;
    return (uint32_t)want;
}

__device__ inline uint64_t g_al256(uint64_t x) { return (x + 255) & ~(uint64_t)255; }

// Appends to the bounded base list.  An append past the capacity is undone,
// so once the appending kernel has finished the count never exceeds the
// capacity and every entry below it is written; the overflow is reported as
// E_NOMEM.
__device__ inline void g_push_base(const GraphArgs &g, uint64_t addr, uint64_t n, uint64_t rlo,
                                   uint64_t rhi) {
    GState *s = g.state;
    const uint32_t q = atomicAdd(&s->base_count, 1u);
    if (q < g.base_cap) {
        g.base_list[4 * q] = addr;
        g.base_list[4 * q + 1] = n;
        g.base_list[4 * q + 2] = rlo;
        g.base_list[4 * q + 3] = rhi;
        atomicAdd(reinterpret_cast<unsigned long long *>(&s->base_elems), (unsigned long long)n);
    } else {
        atomicSub(&s->base_count, 1u);
        set_status(g.lv.status, IPSGPU_E_NOMEM);
    }
}

// Appends to the ring; `floor` is the first entry still in use.
__device__ inline void g_push_ring(const GraphArgs &g, uint64_t floor, const GList &e) {
    unsigned long long *tail = reinterpret_cast<unsigned long long *>(&g.state->tail);
    const uint64_t q = atomicAdd(tail, 1ull);
    if (q - floor < g.ring_cap) {
        g.ring[q % g.ring_cap] = e;
    } else {
        atomicAdd(tail, ~0ull);  // undo
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

// Input arrays fed by a wave that starts with the given state: what is left,
// at most feed_cap (the base list must hold them next to the children of
// the wave) and at most the free ring entries.
__device__ inline uint32_t g_feed_count(const GraphArgs &g, const GJob &j, uint64_t in_head,
                                        uint64_t used) {
    uint64_t f = j.nseg_in > in_head ? j.nseg_in - in_head : 0;
    if (f > g.feed_cap) f = g.feed_cap;
    const uint64_t room = used < g.ring_cap ? g.ring_cap - used : 0;
    if (f > room) f = room;
    return (uint32_t)f;
}

// Starts a run: job and state (one thread).
static __global__ void k_g_job(GraphArgs g, GJob j) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    *g.job = j;
    GState s;
    s.counts = LevelCounts{0, 0, 0, 0, 0, 0};
    s.part_q = 1;
    s.part_blocks = 0;
    s.in_head = 0;
    s.head = 0;
    s.tail = 0;
    s.feed = g_feed_count(g, j, 0, 0);
    s.take = 0;
    s.base_count = 0;
    s.wave = 0;
    s.invalid = 0;
    s.more = 1;
    s.elems = 0;
    s.base_elems = 0;
    s.last_elems = 0;
    s.last_base_elems = 0;
    *g.state = s;
}

// Input arrays [in_head, in_head + feed).  Offsets must be non-decreasing and
// within the data array, listed arrays aligned to the element type; an array
// that is not is skipped, and k_g_advance reports E_INVAL at the end.
static __global__ void __launch_bounds__(256) k_g_feed(GraphArgs g) {
    const GJob j = *g.job;
    const uint64_t i0 = g.state->in_head, i1 = i0 + g.state->feed;
    const uint64_t floor = g.state->head;
    if (j.skip_flags && (j.skip_flags[0] || j.skip_flags[1])) return;  // sorted (or reversed)
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = i0 + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < i1; i += stride) {
        uint64_t addr, n;
        if (j.offsets) {
            const uint64_t b0 = j.offsets[i], b1 = j.offsets[i + 1];
            if (b1 < b0 || b1 > j.n_total) {
                g.state->invalid = 1;
                continue;
            }
            addr = (uint64_t)(uintptr_t)j.data + b0 * g.elem_bytes;
            n = b1 - b0;
        } else if (j.segs) {
            addr = j.segs[2 * i];
            n = j.segs[2 * i + 1];
            if ((n > 0 && (addr == 0 || addr % g.elem_align)) || n > (1ull << 40)) {
                g.state->invalid = 1;
                continue;
            }
        } else {
            addr = (uint64_t)(uintptr_t)j.data;
            n = j.n_total;
        }
        if (n <= 1) continue;
        // radix: the first digit ends at the top key bit, or, when the key
        // range is known, at the highest bit where the smallest and the
        // largest key differ (the bits above are common to every key)
        uint32_t shift = g.keybits > g.kbits ? g.keybits - g.kbits : 0u;
        // an input array's key range is not known (the base case measures
        // it), except for a radix sort's single array, whose detection pass
        // took the smallest and largest key
        uint64_t rlo = ~0ull, rhi = 0;
        if (j.radix_mm && g.algo == 1) {
            const unsigned long long x = j.radix_mm[0] ^ j.radix_mm[1];
            const uint32_t hb = x ? 63u - (uint32_t)__clzll((long long)x) : 0u;
            shift = hb + 1 > g.kbits ? hb + 1 - g.kbits : 0u;
            rlo = j.radix_mm[0];
            rhi = j.radix_mm[1];
        }
        if (n <= g.smax)
            g_push_base(g, addr, n, rlo, rhi);
        else
            g_push_ring(g, floor, GList{addr, n, rlo, rhi, shift, 0u});
    }
}

// Per-segment plan quantities.
struct GPlanItem {
    uint32_t C, p, nc, part0;
    uint64_t arena, sarr, keys, cnt, moves;
};

// Stripe layout of a wave.  Balanced: the wave's blocks, in ring order, are
// cut into parts of Q blocks, one part per classification CTA, and a
// segment's stripes are its pieces of the parts it meets (so every CTA
// classifies the same number of blocks).  Otherwise (a segment too large for
// the arena when cut that way): stripes of about stripe_elems elements,
// classified round-robin.
struct GLayout {
    bool balanced;
    uint64_t Q;             // balanced: blocks per part
    uint64_t stripe_elems;  // otherwise
    uint64_t R;             // virtual permutation CTAs of the window (kPermRounds rounds)
    uint64_t tb;            // blocks waiting in the window
};

// The permutation's virtual CTAs are kPermRounds times the resident ones:
// segments then get kPermRounds times their share of the resident workers
// and run about R / kPermRounds of them at a time.  Measured on 2^30 uint64
// keys (256 segments of 2^22 in the second wave): the wave takes 6.25 ms
// with every segment running at once (3 CTAs each), 4.5 ms with 32 at a
// time; a single segment gets every resident CTA.  Fewer segments at once
// keep fewer bucket fronts open (each bucket's write and read pointers walk
// its region block by block), so DRAM pages and translations are reused.
constexpr uint64_t kPermRounds = 8;

template <class T>
__device__ inline GPlanItem g_item(const GraphArgs &g, uint64_t n, uint64_t gblk0,
                                   const GLayout &ly) {
    GPlanItem it;
    it.C = g.algo == 1 ? (1u << g.kbits) : g_class_budget(g, n);
    const uint64_t nb = (n + g.b - 1) / g.b;
    const uint64_t stage = g_stage_bytes<T>(it.C, g.b), left = g_left_bytes<T>(it.C, g.b);
    uint64_t p;
    it.part0 = 0;
    if (ly.balanced) {
        const uint64_t f = gblk0 / ly.Q, l = (gblk0 + nb - 1) / ly.Q;
        it.part0 = (uint32_t)f;
        p = l - f + 1;
    } else {
        p = (n + ly.stripe_elems - 1) / ly.stripe_elems;
        // one segment alone always fits the arena and the counters (the
        // sorter checks at creation that one stripe of k classes does)
        const uint64_t pfit = g.arena_bytes > stage ? (g.arena_bytes - stage) / left : 1;
        if (p > pfit) p = pfit;
        if (p > g.cnt_cap / it.C) p = g.cnt_cap / it.C;
        if (p > g.stripe_cap) p = g.stripe_cap;
        if (p > nb) p = nb;
        if (p < 1) p = 1;
    }
    // the permutation's virtual CTAs: the window's R shared in proportion
    // to the blocks (a segment gets the CTAs whose share of the block order
    // starts inside it), at least one, at most one per 32 blocks and at most
    // the resident CTAs
    uint64_t nc = (gblk0 + nb) * ly.R / ly.tb - gblk0 * ly.R / ly.tb;
    if (nc > (nb + 31) / 32) nc = (nb + 31) / 32;
    if (nc > g.perm_ctas) nc = g.perm_ctas;
    if (nc > g.cta_cap) nc = g.cta_cap;
    if (nc < 1) nc = 1;
    it.p = (uint32_t)p;
    it.nc = (uint32_t)nc;
    it.arena = stage + p * left;
    it.sarr = seg_arrays_bytes(it.C);
    it.keys = ((uint64_t)2 * it.C * sizeof(typename T::K) + 15) & ~(uint64_t)15;
    it.cnt = (uint64_t)it.C * p;
    it.moves = 2 * ((uint64_t)p + it.C) + 4;
    return it;
}

// Plans the wave: the longest prefix of the ring (at most seg_cap entries)
// whose summed needs fit every capacity.  Stripe and CTA sizes follow the
// elements waiting in the ring window; the balanced layout is tried first.
template <class T>
__global__ void __launch_bounds__(kPlanThreads) k_g_plan(GraphArgs g) {
    constexpr int NV = 9;  // stripes, ctas, classes, arena, sarr, keys, counts, moves, blocks
    __shared__ unsigned long long red[2][32];
    __shared__ unsigned long long wsum[NV][32];
    __shared__ uint32_t sh_cut;
    __shared__ unsigned long long sh_elems;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    GState *S = g.state;
    const uint64_t head = S->head;
    uint64_t avail = S->tail - head;
    uint32_t nin = (uint32_t)(avail < g.seg_cap ? avail : g.seg_cap);
    if (*(volatile int *)g.lv.status != 0) nin = 0;  // an error: stop partitioning
    if (tid == 0) {
        sh_elems = 0;
        *g.lv.nmoves = 0;  // the fix-up moves of this wave start at 0
    }
    // pass 1: elements and blocks waiting in the window
    unsigned long long te = 0, tb = 0;
    for (uint32_t i = tid; i < nin; i += kPlanThreads) {
        const uint64_t n = g.ring[(head + i) % g.ring_cap].n;
        te += n;
        tb += (n + g.b - 1) / g.b;
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
    GLayout ly;
    ly.Q = tb / g.nparts + (tb % g.nparts ? 1 : 0);
    if (ly.Q < 1) ly.Q = 1;
    ly.stripe_elems = te / (2 * (uint64_t)g.nsm);
    if (ly.stripe_elems < kMinStripeElems) ly.stripe_elems = kMinStripeElems;
    ly.stripe_elems = (ly.stripe_elems + g.b - 1) / g.b * g.b;
    ly.R = (g.perm_ctas > 0 ? g.perm_ctas : 1) * kPermRounds;
    ly.tb = tb > 0 ? tb : 1;
    const uint32_t per = (nin + kPlanThreads - 1) / kPlanThreads;
    const uint32_t r0 = min(nin, tid * per), r1 = min(nin, r0 + per);
    const unsigned long long cap[NV] = {g.stripe_cap,  g.cta_cap,    g.cls_cap,
                                        g.arena_bytes, g.sarr_bytes, g.keys_bytes,
                                        g.cnt_cap,     g.lv.move_cap, ~0ull};
    unsigned long long excl[NV];
    uint32_t cut = 0;
    for (int mode = 0; mode < 2; mode++) {
        ly.balanced = mode == 0;
        // block prefix of each thread's range (blocks do not depend on the layout)
        unsigned long long myblk = 0;
        for (uint32_t i = r0; i < r1; i++) myblk += (g.ring[(head + i) % g.ring_cap].n + g.b - 1) / g.b;
        unsigned long long x = myblk;
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        __syncthreads();
        if (lane == 31) wsum[NV - 1][warp] = x;
        __syncthreads();
        unsigned long long gblk = x - myblk;
        for (int w = 0; w < warp; w++) gblk += wsum[NV - 1][w];
        // pass 2: each thread sums its contiguous range of the window
        unsigned long long loc[NV] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        {
            unsigned long long gb = gblk;
            for (uint32_t i = r0; i < r1; i++) {
                const uint64_t n = g.ring[(head + i) % g.ring_cap].n;
                const GPlanItem it = g_item<T>(g, n, gb, ly);
                loc[0] += it.p;
                loc[1] += it.nc;
                loc[2] += it.C;
                loc[3] += it.arena;
                loc[4] += it.sarr;
                loc[5] += it.keys;
                loc[6] += it.cnt;
                loc[7] += it.moves;
                gb += (n + g.b - 1) / g.b;
            }
        }
        loc[8] = myblk;
        __syncthreads();  // every warp has read the block prefix
        // exclusive scan of the sums over threads
#pragma unroll
        for (int v = 0; v < NV; v++) {
            unsigned long long y = loc[v];
            for (int o = 1; o < 32; o <<= 1) {
                unsigned long long z = __shfl_up_sync(0xffffffffu, y, o);
                if (lane >= o) y += z;
            }
            excl[v] = y - loc[v];
            if (lane == 31) wsum[v][warp] = y;
        }
        __syncthreads();
#pragma unroll
        for (int v = 0; v < NV; v++) {
            unsigned long long before = 0;
            for (int w = 0; w < warp; w++) before += wsum[v][w];
            excl[v] += before;
        }
        if (tid == 0) sh_cut = nin;
        __syncthreads();
        // pass 3: the first entry whose running totals exceed a capacity
        {
            unsigned long long run[NV];
#pragma unroll
            for (int v = 0; v < NV; v++) run[v] = excl[v];
            for (uint32_t i = r0; i < r1; i++) {
                const uint64_t n = g.ring[(head + i) % g.ring_cap].n;
                const GPlanItem it = g_item<T>(g, n, run[8], ly);
                run[0] += it.p;
                run[1] += it.nc;
                run[2] += it.C;
                run[3] += it.arena;
                run[4] += it.sarr;
                run[5] += it.keys;
                run[6] += it.cnt;
                run[7] += it.moves;
                run[8] += (n + g.b - 1) / g.b;
                bool over = false;
#pragma unroll
                for (int v = 0; v < NV; v++) over |= run[v] > cap[v];
                if (over) {
                    atomicMin(&sh_cut, i);
                    break;
                }
            }
        }
        __syncthreads();
        cut = sh_cut;
        __syncthreads();
        // a first segment that does not fit when cut into parts: per-segment stripes
        if (cut > 0 || nin == 0) break;
    }
    // pass 4: descriptors of the taken prefix [0, cut)
    unsigned long long my_elems = 0;
    {
        unsigned long long run[NV];
#pragma unroll
        for (int v = 0; v < NV; v++) run[v] = excl[v];
        for (uint32_t i = r0; i < r1 && i < cut; i++) {
            const GList e = g.ring[(head + i) % g.ring_cap];
            const GPlanItem it = g_item<T>(g, e.n, run[8], ly);
            SegDesc d;
            d.addr = e.addr;
            d.n = e.n;
            d.b = g.b;
            d.C = it.C;
            d.stripe0 = (uint32_t)run[0];
            d.nstripes = it.p;
            d.cta0 = (uint32_t)run[1];
            d.ncta = it.nc;
            d.cls0 = (uint32_t)run[2];
            d.stage_off = run[3];
            d.arr_off = run[4];
            d.key_off = run[5];
            d.cnt0 = (uint32_t)run[6];
            d.mode = g.algo == 1 ? 2u : 0u;
            d.radix_shift = e.shift;
            d.radix_bits = g.kbits;
            d.nsplit = 0;
            d.eq_given = 0;
            d.part0 = it.part0;
            d.gblk0 = run[8];
            d.rlo = e.rlo;
            d.rhi = e.rhi;
            const_cast<SegDesc *>(g.lv.seg)[i] = d;
            my_elems += e.n;
            run[0] += it.p;
            run[1] += it.nc;
            run[2] += it.C;
            run[3] += it.arena;
            run[4] += it.sarr;
            run[5] += it.keys;
            run[6] += it.cnt;
            run[7] += it.moves;
            run[8] += (e.n + g.b - 1) / g.b;
            if (i + 1 == cut) {  // the last taken entry knows the totals
                S->counts = LevelCounts{cut,           (uint32_t)run[0], (uint32_t)run[1],
                                        (uint32_t)run[2], ly.balanced ? 1u : 0u, 0u};
                S->part_q = ly.Q;
                S->part_blocks = run[8];
            }
        }
    }
    if (my_elems) atomicAdd(&sh_elems, my_elems);
    __syncthreads();
    if (tid == 0) {
        S->elems = sh_elems;
        S->take = cut;
        if (cut == 0) S->counts = LevelCounts{0, 0, 0, 0, 0, 0};
        if (cut == 0 && nin > 0) set_status(g.lv.status, IPSGPU_E_NOMEM);  // cannot happen
    }
}

// Stripe descriptors, the CTA -> segment map and, for a balanced wave, the
// first stripe of every classification part.
template <class T>
__global__ void __launch_bounds__(256) k_g_fill_stripes(GraphArgs g) {
    const LevelCounts c = g.state->counts;
    const uint64_t Q = g.state->part_q, tblk = g.state->part_blocks;
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
        if (c.balanced) {
            const uint32_t part = sd.part0 + q;
            const uint64_t gb0 = max(sd.gblk0, (uint64_t)part * Q);
            const uint64_t gb1 = min(sd.gblk0 + nb, ((uint64_t)part + 1) * Q);
            s.blk0 = (uint32_t)(gb0 - sd.gblk0);
            s.nblk = (uint32_t)(gb1 - gb0);
            // the first stripe of its part (stripes run in block order)
            if (gb0 == (uint64_t)part * Q || i == 0) g.stripe_first[part] = i;
        } else {
            s.blk0 = (uint32_t)(q * nb / p);
            s.nblk = (uint32_t)((q + 1) * nb / p - q * nb / p);
        }
        s.cnt_off = sd.cnt0 + q * sd.C;
        s.left_off = sd.stage_off + g_stage_bytes<T>(sd.C, sd.b) +
                     (uint64_t)q * g_left_bytes<T>(sd.C, sd.b);
        const_cast<StripeDesc *>(g.lv.stripe)[i] = s;
    }
    if (c.balanced) {
        // parts past the wave's blocks are empty; the end marker
        for (uint32_t part = t0; part <= g.nparts; part += stride)
            if ((uint64_t)part * Q >= tblk) g.stripe_first[part] = c.nstripe;
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

template <class T>
__device__ inline RBounds g_child_bounds(const GraphArgs &g, const SegDesc &sd,
                                         const SegState &st, uint32_t j) {
    const bool known = sd.rlo <= sd.rhi;
    const uint64_t plo = known ? sd.rlo : 0ull, phi = known ? sd.rhi : rk_max<T>();
    if (sd.mode == 2) {  // radix digit j at key bits [shift, shift + bits)
        const uint32_t top = sd.radix_shift + sd.radix_bits;
        const uint64_t above = top >= 64 ? 0ull : ~0ull << top;  // bits common to the parent
        if (!known && above != 0 && top < (uint32_t)g.keybits) return RBounds{~0ull, 0ull};
        const uint64_t lo = (plo & above) | ((uint64_t)j << sd.radix_shift);
        const uint64_t below = sd.radix_shift >= 64 ? ~0ull : ((1ull << sd.radix_shift) - 1);
        return RBounds{lo, lo | below};
    }
    const typename T::K *spl =
        reinterpret_cast<const typename T::K *>(g.lv.keys + sd.key_off) + sd.C;
    const uint32_t K = st.K;
    uint32_t i = j, below_all = 0;
    if (st.eq) {
        i = j >> 1;  // class 2i: s_{i-1} < key < s_i; class 2K - 1: above every splitter
        below_all = j == 2 * K - 1;
    } else {
        below_all = 0;
    }
    uint64_t lo, hi;
    if (below_all) {
        lo = rk_of_key<T>(spl[K - 1]);
        hi = phi;
    } else {
        lo = i == 0 ? plo : rk_of_key<T>(spl[i - 1]);
        hi = i >= K - 1 ? phi : rk_of_key<T>(spl[i]);
    }
    return RBounds{lo, hi};
}

// Children of every (segment, class) of the wave.
template <class T>
__global__ void __launch_bounds__(256) k_g_emit(GraphArgs g) {
    if (*(volatile int *)g.lv.status != 0) return;  // an error: leave the data as is
    const LevelCounts c = g.state->counts;
    const uint64_t floor = g.state->head + g.state->take;  // taken entries are free now
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
        const RBounds rb = g_child_bounds<T>(g, sd, st, j);
        if (n <= g.smax)
            g_push_base(g, sd.addr + b0 * T::D, n, rb.lo, rb.hi);
        else
            g_push_ring(g, floor, GList{sd.addr + b0 * T::D, n, rb.lo, rb.hi, shift, 0u});
    }
}

// Ends a wave (one thread): consumes the taken ring entries and the fed
// inputs, clears the base list, and decides whether another wave runs:
// while inputs or ring entries remain, no error is recorded and the wave
// bound is not reached.  Every wave feeds or partitions at least one
// segment, and children are smaller than their parent (or, for radix, have
// fewer key bits left), so the loop ends; max_waves only guards against an
// inconsistency.  When the run ends, bad inputs become E_INVAL.
static __global__ void k_g_advance(GraphArgs g, cudaGraphConditionalHandle h, int in_graph) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    GState *S = g.state;
    const GJob j = *g.job;
    S->head += S->take;
    S->in_head += S->feed;
    S->take = 0;
    S->base_count = 0;
    S->last_elems = S->elems;
    S->last_base_elems = S->base_elems;
    S->elems = 0;
    S->base_elems = 0;
    S->counts = LevelCounts{0, 0, 0, 0, 0, 0};
    S->wave += 1;
    const bool work = S->in_head < j.nseg_in || S->head < S->tail;
    const int status = *(volatile int *)g.lv.status;
    uint32_t more = (work && status == 0) ? 1u : 0u;
    if (more && S->wave >= j.max_waves) {
        set_status(g.lv.status, IPSGPU_E_INTERNAL);
        more = 0;
    }
    S->feed = more ? g_feed_count(g, j, S->in_head, S->tail - S->head) : 0u;
    if (!more && S->invalid) set_status(g.lv.status, IPSGPU_E_INVAL);
    S->more = more;
    if (in_graph) cudaGraphSetConditional(h, more);
}

}  // namespace ipsgpu

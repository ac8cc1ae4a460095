// ipsgpu.cu -- the C ABI (include/ipsgpu.h) on the host side: parameter
// resolution and scratch (with guard zones), easy-input detection, the CUDA
// graph that runs the device-planned recursion (graph.cuh: waves over all
// pending segments, Sec. 3.2 task structure breadth-first, Sec. 5
// parameters) or its host-driven twin when kernels are timed, host-planned
// single levels (partition_level, radix_level, classify), batched and
// segmented runs, and the host-array call.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <utility>
#include <vector>

#include "graph.cuh"
#include "sorter.h"

using namespace ipsgpu;

struct ipsgpu_sorter {
    Sorter s;
};

namespace {

constexpr uint64_t kMinStripe = 1u << 15;  // elements
// shared memory one CTA may opt in to on sm_100 / sm_103 GPUs (227 KiB)
constexpr uint64_t kSmemOptinBytes = 227u * 1024;
constexpr uint64_t kStaticSmemSlack = 1024;  // a kernel's static shared variables

__global__ void k_debug_wait(uint32_t *flag, uint32_t limit, int *status) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        if (!bounded_wait_eq(flag, 1u, limit)) set_status(status, IPSGPU_E_TIMEOUT);
    }
}

const TypeOps *ops_for(int dtype) {
    switch (dtype) {
    case IPSGPU_U32: return &ops_u32;
    case IPSGPU_U64: return &ops_u64;
    case IPSGPU_F64: return &ops_f64;
    case IPSGPU_PAIR_U64: return &ops_pair;
    case IPSGPU_REC100: return &ops_rec100;
    case IPSGPU_QUARTET: return &ops_quartet;
    default: return nullptr;
    }
}

uint64_t next_pow2(uint64_t x) {
    uint64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

uint64_t align_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

// alignment the kernels need of a data array: the element size (4 bytes for
// rec100), at most 16
uint64_t elem_align(int D) { return D == 100 ? 4 : (uint64_t)std::min(D, 16); }

// block size in elements: block_bytes / D rounded down to a power of two
uint32_t block_elems(uint32_t block_bytes, int D) {
    uint32_t b = 1;
    while ((uint64_t)b * 2 * D <= block_bytes) b *= 2;
    return b;
}

struct Resolved {
    uint32_t k, block_bytes, base_case, spin_limit;
    float alpha_scale;
    uint64_t seed, arena_bytes;
    int algo;
};

int resolve(const ipsgpu_params *p, int dtype, Resolved *r) {
    const TypeOps *ops = ops_for(dtype);
    if (!ops) return IPSGPU_E_INVAL;
    r->k = (p && p->k) ? p->k : 256;
    r->block_bytes = (p && p->block_bytes) ? p->block_bytes : 512;
    r->alpha_scale = (p && p->alpha_scale > 0) ? p->alpha_scale : 0.2f;
    r->seed = (p && p->seed) ? p->seed : 0x1B54A32D192ED03ull;
    r->algo = p ? p->algo : IPSGPU_SAMPLESORT;
    r->spin_limit = (p && p->spin_limit) ? p->spin_limit : (1u << 22);
    r->arena_bytes = (p && p->arena_bytes) ? p->arena_bytes : (256ull << 20);
    const uint32_t cap = (uint32_t)(kBaseSmemBytes / ops->D);
    r->base_case = (p && p->base_case) ? p->base_case : cap;
    if (r->k < 4 || r->k > (uint32_t)kMaxClasses || (r->k & (r->k - 1))) return IPSGPU_E_INVAL;
    if (r->base_case < 32 || r->base_case > cap) return IPSGPU_E_INVAL;
    // blocks: a multiple of 16 bytes, at most kMaxBlockBytes (a permutation
    // worker holds one in registers); k of them plus the tile stage fit the
    // shared memory of one classification CTA
    uint32_t b = block_elems(r->block_bytes, ops->D);
    if (b == 0 || (uint64_t)b * ops->D > kMaxBlockBytes || (b * ops->D) % 16 ||
        ops->classify_smem_bytes(r->k, b) + kStaticSmemSlack > kSmemOptinBytes)
        return IPSGPU_E_INVAL;
    // the arena holds at least one segment with one stripe of k classes
    if (r->arena_bytes < 2ull * r->k * b * ops->D + (uint64_t)b * ops->D + 1024) return IPSGPU_E_INVAL;
    if (r->algo != IPSGPU_SAMPLESORT && r->algo != IPSGPU_RADIX &&
        r->algo != IPSGPU_SAMPLESORT_TREE)
        return IPSGPU_E_INVAL;
    if (r->algo == IPSGPU_RADIX &&
        !(dtype == IPSGPU_U32 || dtype == IPSGPU_U64 || dtype == IPSGPU_PAIR_U64))
        return IPSGPU_E_UNSUPPORTED;
    return IPSGPU_OK;
}

struct Layout {
    uint64_t seg, st, sarr, keys, stripe, scount, sfull, arena, moves, cta, base, ring, misc;
    uint64_t total() const {
        return seg + st + sarr + keys + stripe + scount + sfull + arena + moves + cta + base + ring +
               misc;
    }
};

// Per-segment sizes: SegArrays of C classes fit 28 C + 32 bytes, the tree
// and splitters 2 C keys + 16 bytes; both summed over at most cls_cap
// classes and seg_cap segments.
Layout layout(const Sorter &s, int key_bytes) {
    Layout L;
    L.seg = (uint64_t)s.seg_cap * sizeof(SegDesc);
    L.st = (uint64_t)s.seg_cap * sizeof(SegState);
    L.sarr = (uint64_t)28 * s.cls_cap + 32ull * s.seg_cap;
    L.keys = (uint64_t)2 * s.cls_cap * key_bytes + 16ull * s.seg_cap;
    L.stripe = (uint64_t)s.stripe_cap * sizeof(StripeDesc);
    L.scount = (uint64_t)s.cnt_cap * sizeof(uint32_t);
    L.sfull = (uint64_t)s.stripe_cap * sizeof(uint32_t);
    L.arena = s.arena_bytes;
    L.moves = (uint64_t)s.move_cap * sizeof(Move);
    L.cta = (uint64_t)s.cta_cap * sizeof(uint32_t);
    L.base = (uint64_t)s.base_cap * 4 * sizeof(uint64_t);
    L.ring = (uint64_t)s.ring_cap * sizeof(GList);
    L.misc = 1024;
    return L;
}

void apply(Sorter &s, const Resolved &r, int dtype) {
    s.dtype = dtype;
    s.ops = ops_for(dtype);
    s.k = r.k;
    s.block_bytes = r.block_bytes;
    s.alpha_scale = r.alpha_scale;
    s.seed = r.seed;
    s.algo = r.algo;
    s.spin_limit = r.spin_limit;
    s.arena_bytes = r.arena_bytes;
    s.b = block_elems(r.block_bytes, s.ops->D);
    s.smax = r.base_case;
    Layout L = layout(s, s.ops->key_bytes);
    s.sarr_bytes = L.sarr;
    s.keys_bytes = L.keys;
}

int cuda_status(cudaError_t e) { return e == cudaSuccess ? IPSGPU_OK : IPSGPU_E_CUDA; }

void free_all(Sorter &s) {
    for (const auto &g : s.guarded) cudaFree(g.base);
    s.guarded.clear();
    if (s.wave_exec) cudaGraphExecDestroy(s.wave_exec);
    if (s.wave_graph) cudaGraphDestroy(s.wave_graph);
    if (s.cap_stream) cudaStreamDestroy(s.cap_stream);
    void *host[] = {s.h_seg, s.h_stripe, s.h_cta_seg, s.h_flags, s.h_gstate};
    for (void *p : host)
        if (p) cudaFreeHost(p);
    for (auto &l : s.launches) {
        cudaEventDestroy(l.ev0);
        cudaEventDestroy(l.ev1);
    }
    for (auto e : s.event_pool) cudaEventDestroy(e);
    if (s.h2d_done) cudaEventDestroy(s.h2d_done);
}

// ------------------------------------------------------------------ levels
struct Pending {
    uint64_t addr, n;  // device byte address of the first element, elements
    uint32_t shift;    // radix: the digit to use is bits [shift, shift+bits)
};

struct BatchPlan {
    uint32_t nseg = 0, nstripe = 0, ncta = 0, nmoves = 0, ncls = 0, ncnt = 0;
    uint64_t arena = 0, elems = 0, sarr = 0, keys = 0;
};

// Plans one segment of a single partitioning step (given splitters or one
// radix digit) into the pinned descriptors.
int plan_single(Sorter &s, const Pending &pd, uint32_t mode, uint32_t nsplit, int eq_given,
                uint32_t radix_bits, uint64_t stripe_elems, uint64_t blocks_per_cta,
                BatchPlan &bp) {
    const uint64_t D = s.ops->D;
    uint32_t C;
    if (mode == 1) {
        uint64_t K = next_pow2((uint64_t)nsplit + 1);
        C = (uint32_t)(eq_given ? 2 * K : K);
    } else {
        C = 1u << radix_bits;
    }
    const uint64_t nb = (pd.n + s.b - 1) / s.b;
    uint64_t p = (pd.n + stripe_elems - 1) / stripe_elems;
    if (p < 1) p = 1;
    if (p > nb) p = nb;
    uint64_t nc = (nb + blocks_per_cta - 1) / blocks_per_cta;
    if (nc < 1) nc = 1;
    // arena: cleanup staging (C blocks) directly followed by the overflow
    // block, then C leftover buffer blocks per stripe
    const uint64_t stageb = align_up((uint64_t)C * s.b * D + (uint64_t)s.b * D, 256);
    const uint64_t bufb = align_up((uint64_t)C * s.b * D, 256);
    if (p > s.stripe_cap || nc > s.cta_cap || stageb + p * bufb > s.arena_bytes ||
        2 * (p + C) + 4 > s.move_cap || (uint64_t)C * p > s.cnt_cap)
        return IPSGPU_E_NOMEM;
    SegDesc &sd = s.h_seg[0];
    memset(&sd, 0, sizeof sd);
    sd.addr = pd.addr;
    sd.n = pd.n;
    sd.b = s.b;
    sd.C = C;
    sd.stripe0 = 0;
    sd.nstripes = (uint32_t)p;
    sd.cta0 = 0;
    sd.ncta = (uint32_t)nc;
    sd.stage_off = 0;
    sd.arr_off = 0;
    sd.key_off = 0;
    sd.cls0 = 0;
    sd.cnt0 = 0;
    sd.mode = mode;
    sd.radix_shift = pd.shift;
    sd.radix_bits = radix_bits;
    sd.nsplit = nsplit;
    sd.eq_given = eq_given ? 1 : 0;
    uint64_t off = stageb;
    for (uint64_t q = 0; q < p; q++) {
        StripeDesc &sp = s.h_stripe[q];
        sp.seg = 0;
        const uint64_t b0 = q * nb / p, b1 = (q + 1) * nb / p;
        sp.blk0 = (uint32_t)b0;
        sp.nblk = (uint32_t)(b1 - b0);
        sp.cnt_off = (uint32_t)(q * C);
        sp.left_off = off;
        off += bufb;
    }
    for (uint64_t c = 0; c < nc; c++) s.h_cta_seg[c] = 0;
    bp.nseg = 1;
    bp.nstripe = (uint32_t)p;
    bp.ncta = (uint32_t)nc;
    bp.ncls = C;
    bp.elems = pd.n;
    return IPSGPU_OK;
}

int upload_plan(Sorter &s, const BatchPlan &bp, cudaStream_t st) {
    cudaError_t e;
    e = cudaMemcpyAsync(s.d_seg, s.h_seg, sizeof(SegDesc) * bp.nseg, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && bp.nstripe)
        e = cudaMemcpyAsync(s.d_stripe, s.h_stripe, sizeof(StripeDesc) * bp.nstripe,
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && bp.ncta)
        e = cudaMemcpyAsync(s.d_cta_seg, s.h_cta_seg, sizeof(uint32_t) * bp.ncta,
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaEventRecord(s.h2d_done, st);
    return cuda_status(e);
}

// the pinned mirrors may be rewritten only once earlier uploads have run
int wait_uploads(Sorter &s) { return cuda_status(cudaEventSynchronize(s.h2d_done)); }

// stripes of about n / (2 * #SM) elements (at least kMinStripe), and about
// 8 block-permutation CTAs per SM (at least 32 blocks each); the device
// planner uses the same rule over a level's total
void level_sizes(const Sorter &s, uint64_t tot, uint64_t &stripe_elems, uint64_t &blocks_per_cta) {
    const uint64_t blocks = (tot + s.b - 1) / s.b;
    stripe_elems = std::max<uint64_t>(kMinStripe, tot / (2 * (uint64_t)s.nsm));
    stripe_elems = align_up(stripe_elems, s.b);
    // one virtual permutation CTA per resident CTA
    const uint64_t pc = std::max<uint64_t>(1, s.perm_ctas);
    blocks_per_cta = std::max<uint64_t>(32, (blocks + pc - 1) / pc);
}

int read_status(Sorter &s, cudaStream_t st, int *code) {
    cudaError_t e = cudaMemcpyAsync(s.h_flags + 2, s.d_status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return IPSGPU_E_CUDA;
    *code = s.h_flags[2];
    return IPSGPU_OK;
}

int check_data(const Sorter &s, const void *d) {
    if (!d) return IPSGPU_E_INVAL;
    return ((uintptr_t)d % elem_align(s.ops->D)) ? IPSGPU_E_INVAL : IPSGPU_OK;
}

// Fixed arguments of the device-planned recursion of this sorter.
GraphArgs graph_args(Sorter &s) {
    GraphArgs ga;
    memset(&ga, 0, sizeof ga);
    ga.lv = s.args(0, 0, 0, 0, nullptr);
    ga.job = reinterpret_cast<GJob *>(s.d_gjob);
    ga.state = reinterpret_cast<GState *>(s.d_gstate);
    ga.lv.cnt = &ga.state->counts;
    ga.ring = reinterpret_cast<GList *>(s.d_ring);
    ga.base_list = s.d_base;
    ga.stripe_first = s.d_stripe_first;
    ga.nparts = (uint32_t)s.nsm;
    ga.ring_cap = s.ring_cap;
    ga.base_cap = s.base_cap;
    ga.feed_cap = s.base_cap - s.cls_cap;
    ga.seg_cap = s.seg_cap;
    ga.stripe_cap = s.stripe_cap;
    ga.cta_cap = s.cta_cap;
    ga.cls_cap = s.cls_cap;
    ga.cnt_cap = s.cnt_cap;
    ga.smax = s.smax;
    ga.k = s.k;
    ga.b = s.b;
    ga.nsm = (uint32_t)s.nsm;
    ga.perm_ctas = s.perm_ctas;
    ga.kbits = (uint32_t)__builtin_ctz(s.k);
    ga.keybits = s.ops->D == 4 ? 32 : 64;
    ga.elem_bytes = (uint32_t)s.ops->D;
    ga.elem_align = (uint32_t)elem_align(s.ops->D);
    ga.arena_bytes = s.arena_bytes;
    ga.sarr_bytes = s.sarr_bytes;
    ga.keys_bytes = s.keys_bytes;
    ga.algo = s.algo == IPSGPU_RADIX ? 1 : 0;
    return ga;
}

// Bound on the waves of one run; the loop ends by itself long before (every
// wave makes progress), the bound only stops an inconsistent run.
constexpr uint32_t kMaxWaves = 1u << 20;

// Builds a graph that runs waves while k_g_advance says so: an optional
// k_g_job node (the run's input) followed by a conditional WHILE node whose
// body is one wave.
int build_wave_graph(Sorter &s, const GJob *job, cudaGraph_t *out_graph, cudaGraphExec_t *out_exec) {
    *out_graph = nullptr;
    *out_exec = nullptr;
    if (!s.cap_stream &&
        cudaStreamCreateWithFlags(&s.cap_stream, cudaStreamNonBlocking) != cudaSuccess)
        return IPSGPU_E_CUDA;
    const GraphArgs ga = graph_args(s);
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ex = nullptr;
    const bool timing = s.timing;
    s.timing = false;  // no event records inside a graph
    int rc = IPSGPU_OK;
    do {
        if (cudaGraphCreate(&g, 0) != cudaSuccess) { rc = IPSGPU_E_CUDA; break; }
        cudaGraphNode_t jobnode = nullptr;
        if (job) {
            if (cudaStreamBeginCaptureToGraph(s.cap_stream, g, nullptr, nullptr, 0,
                                              cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
                rc = IPSGPU_E_CUDA;
                break;
            }
            k_g_job<<<1, 32, 0, s.cap_stream>>>(ga, *job);
            cudaGraph_t g2 = nullptr;
            if (cudaStreamEndCapture(s.cap_stream, &g2) != cudaSuccess) { rc = IPSGPU_E_CUDA; break; }
            size_t nn = 1;
            if (cudaGraphGetNodes(g, &jobnode, &nn) != cudaSuccess || nn != 1) {
                rc = IPSGPU_E_CUDA;
                break;
            }
        }
        cudaGraphConditionalHandle h;
        if (cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) != cudaSuccess) {
            rc = IPSGPU_E_CUDA;
            break;
        }
        cudaGraphNodeParams p = {};
        p.type = cudaGraphNodeTypeConditional;
        p.conditional.handle = h;
        p.conditional.type = cudaGraphCondTypeWhile;
        p.conditional.size = 1;
        cudaGraphNode_t cond;
        if (cudaGraphAddNode(&cond, g, job ? &jobnode : nullptr, nullptr, job ? 1 : 0, &p) !=
            cudaSuccess) {
            rc = IPSGPU_E_CUDA;
            break;
        }
        cudaGraph_t body = p.conditional.phGraph_out[0];
        if (cudaStreamBeginCaptureToGraph(s.cap_stream, body, nullptr, nullptr, 0,
                                          cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            rc = IPSGPU_E_CUDA;
            break;
        }
        rc = cuda_status(s.ops->wave(&s, ga, s.cap_stream, 1, h));
        cudaGraph_t body2 = nullptr;
        if (cudaStreamEndCapture(s.cap_stream, &body2) != cudaSuccess && rc == IPSGPU_OK)
            rc = IPSGPU_E_CUDA;
        if (rc) break;
        if (cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) rc = IPSGPU_E_CUDA;
    } while (0);
    s.timing = timing;
    if (rc) {
        if (ex) cudaGraphExecDestroy(ex);
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return rc;
    }
    *out_graph = g;
    *out_exec = ex;
    return IPSGPU_OK;
}

// One device-planned run (graph.cuh) over `job`: the sorter's WHILE graph
// after a k_g_job launch, or, with per-kernel timing on, the same waves from
// a host loop (one synchronization per wave to read the decision back).
int graph_run(Sorter &s, const GJob &job, cudaStream_t st) {
    const GraphArgs ga = graph_args(s);
    k_g_job<<<1, 32, 0, st>>>(ga, job);
    if (cudaGetLastError() != cudaSuccess) return IPSGPU_E_CUDA;
    if (!s.timing) {
        if (!s.wave_exec) {
            int rc = build_wave_graph(s, nullptr, &s.wave_graph, &s.wave_exec);
            if (rc) return rc;
        }
        return cuda_status(cudaGraphLaunch(s.wave_exec, st));
    }
    s.last_waves = 0;
    s.last_max_pending = 0;
    for (uint32_t w = 0; w < kMaxWaves; w++) {
        NvtxRange nvtx_wave("ipsgpu wave");
        const size_t l0 = s.launches.size();
        cudaError_t e = s.ops->wave(&s, ga, st, 0, cudaGraphConditionalHandle());
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(s.h_gstate, ga.state, sizeof(GState), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return IPSGPU_E_CUDA;
        const GState &gs = *reinterpret_cast<const GState *>(s.h_gstate);
        s.last_waves++;
        s.last_max_pending = std::max<uint64_t>(s.last_max_pending, gs.tail - gs.head);
        // algorithmic bytes of the wave's launches (2 D per element moved)
        for (size_t q = l0; q < s.launches.size(); q++) {
            TimedLaunch &l = s.launches[q];
            if (l.kind == KK_CLASSIFY || l.kind == KK_PERMUTE)
                l.bytes = 2.0 * (double)gs.last_elems * s.ops->D;
            else if (l.kind == KK_BASE)
                l.bytes = 2.0 * (double)gs.last_base_elems * s.ops->D;
        }
        if (!gs.more) break;
    }
    return IPSGPU_OK;
}

GJob make_job(unsigned char *data, uint64_t n_total, const uint64_t *offsets, const uint64_t *segs,
              uint64_t nseg, const int *skip_flags, const unsigned long long *radix_mm = nullptr) {
    GJob j;
    memset(&j, 0, sizeof j);
    j.data = data;
    j.offsets = offsets;
    j.segs = segs;
    j.skip_flags = skip_flags;
    j.radix_mm = radix_mm;
    j.nseg_in = nseg;
    j.n_total = n_total;
    j.max_waves = kMaxWaves;
    return j;
}

// The whole sort on the device (no host synchronization): Sec. 5's check for
// non-decreasing and non-increasing inputs (one pass, flags in device
// memory; a non-increasing input is reversed), then the recursion, skipped
// when a flag is set.
int sort_impl(Sorter &s, unsigned char *data, uint64_t n, cudaStream_t st) {
    if (n < 2) return IPSGPU_OK;
    if (n > (1ull << 40)) return IPSGPU_E_INVAL;
    s.data = data;
    // both flags start non-zero ("still possible"); for radix the key
    // min / max words follow them (d_flags + 2: ~0, then 0)
    const bool radix = s.algo == IPSGPU_RADIX;
    unsigned long long *mm = reinterpret_cast<unsigned long long *>(s.d_flags + 2);
    cudaError_t e = cudaMemsetAsync(s.d_flags, 1, 2 * sizeof(int), st);
    if (e == cudaSuccess && radix) e = cudaMemsetAsync(mm, 0xFF, sizeof(unsigned long long), st);
    if (e == cudaSuccess && radix) e = cudaMemsetAsync(mm + 1, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = s.ops->detect(&s, data, n, radix ? mm : nullptr, st);
    if (e == cudaSuccess) e = s.ops->reverse(&s, data, n, st);
    if (e != cudaSuccess) return IPSGPU_E_CUDA;
    s.level_elems = n;
    return graph_run(s, make_job(data, n, nullptr, nullptr, 1, s.d_flags, radix ? mm : nullptr), st);
}

int single_level(Sorter &s, unsigned char *data, uint64_t n, uint32_t mode, uint32_t nsplit,
                 int eq, uint32_t shift, uint32_t bits, const unsigned char *given,
                 cudaStream_t st) {
    s.data = data;
    int rc = wait_uploads(s);
    if (rc) return rc;
    uint64_t stripe_elems, bpc;
    level_sizes(s, n, stripe_elems, bpc);
    BatchPlan bp;
    rc = plan_single(s, Pending{(uint64_t)(uintptr_t)data, n, shift}, mode, nsplit, eq, bits,
                     stripe_elems, bpc, bp);
    if (rc) return rc;
    if ((rc = upload_plan(s, bp, st))) return rc;
    s.level_elems = n;
    const LevelArgs a = s.args(bp.nseg, bp.nstripe, bp.ncta, bp.ncls, given);
    const LevelGrids g{bp.nseg, bp.nstripe, bp.ncta, bp.ncls};
    return cuda_status(s.ops->level(&s, a, g, st));
}

}  // namespace

// ------------------------------------------------------------- Sorter methods
namespace ipsgpu {

LevelArgs Sorter::args(uint32_t nseg, uint32_t nstripe, uint32_t ncta, uint32_t ncls,
                       const unsigned char *given_spl) const {
    LevelArgs a;
    memset(&a, 0, sizeof a);
    a.data = data;
    a.seg = d_seg;
    a.st = d_st;
    a.sarr = d_sarr;
    a.keys = d_keys;
    a.given_spl = given_spl;
    a.stripe = d_stripe;
    a.scount = d_scount;
    a.sfull = d_sfull;
    a.arena = d_arena;
    a.moves = d_moves;
    a.nmoves = d_nmoves;
    a.move_cap = move_cap;
    a.status = d_status;
    a.nseg = nseg;
    a.nstripe = nstripe;
    a.ncta = ncta;
    a.ncls = ncls;
    a.cnt = nullptr;
    a.cta_seg = d_cta_seg;
    a.spin_limit = spin_limit;
    a.tree_only = algo == IPSGPU_SAMPLESORT_TREE ? 1u : 0u;
    a.seed = seed;
    a.alpha_scale = alpha_scale;
    return a;
}

void Sorter::tbegin(int kind, double bytes, cudaStream_t st) {
    if (!timing) return;
    TimedLaunch l;
    l.kind = kind;
    l.bytes = bytes;
    for (int q = 0; q < 2; q++) {
        cudaEvent_t ev;
        if (!event_pool.empty()) {
            ev = event_pool.back();
            event_pool.pop_back();
        } else {
            cudaEventCreate(&ev);
        }
        (q == 0 ? l.ev0 : l.ev1) = ev;
    }
    cudaEventRecord(l.ev0, st);
    launches.push_back(l);
}

void Sorter::tend(cudaStream_t st) {
    if (!timing || launches.empty()) return;
    cudaEventRecord(launches.back().ev1, st);
}

void Sorter::collect() {
    for (auto &l : launches) {
        float ms = 0.f;
        cudaEventSynchronize(l.ev1);
        cudaEventElapsedTime(&ms, l.ev0, l.ev1);
        stat_launches[l.kind]++;
        stat_ms[l.kind] += ms;
        stat_bytes[l.kind] += l.bytes;
        event_pool.push_back(l.ev0);
        event_pool.push_back(l.ev1);
    }
    launches.clear();
}

}  // namespace ipsgpu

// ------------------------------------------------------------------ C ABI
extern "C" {

uint64_t ipsgpu_scratch_bytes(const ipsgpu_params *params, int dtype) {
    Resolved r;
    if (resolve(params, dtype, &r) != IPSGPU_OK) return 0;
    Sorter s;
    apply(s, r, dtype);
    return layout(s, s.ops->key_bytes).total();
}

int ipsgpu_sorter_create(const ipsgpu_params *params, int dtype, ipsgpu_sorter **out) {
    NvtxRange nvtx_range("ipsgpu_sorter_create");
    if (!out) return IPSGPU_E_INVAL;
    *out = nullptr;
    Resolved r;
    int rc = resolve(params, dtype, &r);
    if (rc) return rc;
    ipsgpu_sorter *h = new (std::nothrow) ipsgpu_sorter;
    if (!h) return IPSGPU_E_NOMEM;
    Sorter &s = h->s;
    apply(s, r, dtype);
    if (cudaGetDevice(&s.device) != cudaSuccess ||
        cudaDeviceGetAttribute(&s.nsm, cudaDevAttrMultiProcessorCount, s.device) != cudaSuccess) {
        delete h;
        return IPSGPU_E_CUDA;
    }
    Layout L = layout(s, s.ops->key_bytes);
    s.scratch_bytes = L.total();
    bool ok = true;
    // device buffers between guard zones (see Sorter::guarded)
    auto dm = [&](void **p, uint64_t bytes) {
        if (!ok) return;
        if (!bytes) bytes = 16;
        unsigned char *base = nullptr;
        if (cudaMalloc((void **)&base, bytes + 2 * kGuardBytes) != cudaSuccess) {
            ok = false;
            return;
        }
        s.guarded.push_back({base, bytes});
        if (cudaMemset(base, kGuardByte, kGuardBytes) != cudaSuccess ||
            cudaMemset(base + kGuardBytes + bytes, kGuardByte, kGuardBytes) != cudaSuccess)
            ok = false;
        *p = base + kGuardBytes;
    };
    auto hm = [&](void **p, uint64_t bytes) {
        if (ok && cudaMallocHost(p, bytes ? bytes : 16) != cudaSuccess) ok = false;
    };
    dm((void **)&s.d_seg, L.seg);
    dm((void **)&s.d_st, L.st);
    dm((void **)&s.d_sarr, L.sarr);
    dm((void **)&s.d_keys, L.keys);
    dm((void **)&s.d_stripe, L.stripe);
    dm((void **)&s.d_scount, L.scount);
    dm((void **)&s.d_sfull, L.sfull);
    dm((void **)&s.d_arena, L.arena);
    dm((void **)&s.d_moves, L.moves);
    dm((void **)&s.d_nmoves, 64);
    dm((void **)&s.d_status, 64);
    dm((void **)&s.d_cta_seg, L.cta);
    dm((void **)&s.d_base, L.base);
    dm((void **)&s.d_flags, 64);
    dm((void **)&s.d_waitflag, 64);
    dm((void **)&s.d_ring, L.ring);
    dm((void **)&s.d_stripe_first, sizeof(uint32_t) * 4096);
    dm((void **)&s.d_gjob, 256);
    dm((void **)&s.d_gstate, 256);
    hm((void **)&s.h_seg, L.seg);
    hm((void **)&s.h_stripe, L.stripe);
    hm((void **)&s.h_cta_seg, L.cta);
    hm((void **)&s.h_flags, 64);
    hm((void **)&s.h_gstate, 256);
    if (ok && cudaEventCreateWithFlags(&s.h2d_done, cudaEventDisableTiming) != cudaSuccess) ok = false;
    if (ok && (cudaMemset(s.d_status, 0, 64) != cudaSuccess ||
               cudaMemset(s.d_waitflag, 0, 64) != cudaSuccess))
        ok = false;
    if (ok && s.ops->init(&s) != cudaSuccess) {
        free_all(s);
        delete h;
        return IPSGPU_E_CUDA;
    }
    if (!ok) {
        free_all(s);
        delete h;
        cudaGetLastError();
        return IPSGPU_E_NOMEM;
    }
    if (cudaEventRecord(s.h2d_done, 0) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
        free_all(s);
        delete h;
        return IPSGPU_E_CUDA;
    }
    *out = h;
    return IPSGPU_OK;
}

int ipsgpu_debug_check_guards(ipsgpu_sorter *h, uint64_t *first_bad) {
    if (!h) return IPSGPU_E_INVAL;
    Sorter &s = h->s;
    if (cudaDeviceSynchronize() != cudaSuccess) return IPSGPU_E_CUDA;
    std::vector<unsigned char> buf(2 * kGuardBytes);
    for (size_t i = 0; i < s.guarded.size(); i++) {
        const auto &g = s.guarded[i];
        if (cudaMemcpy(buf.data(), g.base, kGuardBytes, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(buf.data() + kGuardBytes, g.base + kGuardBytes + g.bytes, kGuardBytes,
                       cudaMemcpyDeviceToHost) != cudaSuccess)
            return IPSGPU_E_CUDA;
        for (unsigned char c : buf) {
            if (c != kGuardByte) {
                if (first_bad) *first_bad = (uint64_t)i;
                return IPSGPU_E_INTERNAL;
            }
        }
    }
    if (first_bad) *first_bad = ~0ull;
    return IPSGPU_OK;
}

int ipsgpu_sorter_prepare(ipsgpu_sorter *h) {
    NvtxRange nvtx_range("ipsgpu_sorter_prepare");
    if (!h) return IPSGPU_E_INVAL;
    Sorter &s = h->s;
    if (s.wave_exec) return IPSGPU_OK;
    return build_wave_graph(s, nullptr, &s.wave_graph, &s.wave_exec);
}

int ipsgpu_sorter_destroy(ipsgpu_sorter *h) {
    if (!h) return IPSGPU_E_INVAL;
    cudaDeviceSynchronize();
    free_all(h->s);
    delete h;
    return IPSGPU_OK;
}

int ipsgpu_sort(ipsgpu_sorter *h, void *d_data, uint64_t n, void *stream) {
    NvtxRange nvtx_range("ipsgpu_sort");
    if (!h) return IPSGPU_E_INVAL;
    if (n == 0) return IPSGPU_OK;
    int rc = check_data(h->s, d_data);
    if (rc) return rc;
    return sort_impl(h->s, (unsigned char *)d_data, n, (cudaStream_t)stream);
}

int ipsgpu_sort_host(ipsgpu_sorter *h, const void *h_in, void *h_out, uint64_t n, void *d_work,
                     void *stream) {
    NvtxRange nvtx_range("ipsgpu_sort_host");
    if (!h || !h_in || !h_out) return IPSGPU_E_INVAL;
    if (n == 0) return IPSGPU_OK;
    Sorter &s = h->s;
    int rc = check_data(s, d_work);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = (size_t)n * s.ops->D;
    if (cudaMemcpyAsync(d_work, h_in, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return IPSGPU_E_CUDA;
    if ((rc = sort_impl(s, (unsigned char *)d_work, n, st))) return rc;
    return cuda_status(cudaMemcpyAsync(h_out, d_work, bytes, cudaMemcpyDeviceToHost, st));
}

int ipsgpu_partition_level(ipsgpu_sorter *h, void *d_data, uint64_t n, const void *d_splitters,
                           uint32_t num_splitters, int equal_buckets, uint64_t *d_bucket_begin,
                           void *stream) {
    NvtxRange nvtx_range("ipsgpu_partition_level");
    if (!h || !d_bucket_begin || !d_splitters || num_splitters == 0) return IPSGPU_E_INVAL;
    Sorter &s = h->s;
    const uint64_t K = next_pow2((uint64_t)num_splitters + 1);
    const uint64_t B = equal_buckets ? 2 * K : K;
    if (B > s.k) return IPSGPU_E_INVAL;
    cudaStream_t st = (cudaStream_t)stream;
    if (n == 0)
        return cuda_status(cudaMemsetAsync(d_bucket_begin, 0, sizeof(uint64_t) * (B + 1), st));
    int rc = check_data(s, d_data);
    if (rc || (rc = check_data(s, d_splitters))) return rc;
    rc = single_level(s, (unsigned char *)d_data, n, 1, num_splitters, equal_buckets, 0, 0,
                      (const unsigned char *)d_splitters, st);
    if (rc) return rc;
    // the single segment's SegArrays start the state arena: bucket_begin first
    return cuda_status(cudaMemcpyAsync(d_bucket_begin, s.d_sarr, sizeof(uint64_t) * (B + 1),
                                       cudaMemcpyDeviceToDevice, st));
}

int ipsgpu_radix_level(ipsgpu_sorter *h, void *d_data, uint64_t n, uint32_t shift, uint32_t bits,
                       uint64_t *d_bucket_begin, void *stream) {
    NvtxRange nvtx_range("ipsgpu_radix_level");
    if (!h || !d_bucket_begin) return IPSGPU_E_INVAL;
    Sorter &s = h->s;
    if (!(s.dtype == IPSGPU_U32 || s.dtype == IPSGPU_U64 || s.dtype == IPSGPU_PAIR_U64))
        return IPSGPU_E_UNSUPPORTED;
    const uint32_t keybits = s.dtype == IPSGPU_U32 ? 32 : 64;
    if (bits < 1 || bits > 8 || (1u << bits) > s.k || shift >= keybits) return IPSGPU_E_INVAL;
    const uint64_t B = 1ull << bits;
    cudaStream_t st = (cudaStream_t)stream;
    if (n == 0)
        return cuda_status(cudaMemsetAsync(d_bucket_begin, 0, sizeof(uint64_t) * (B + 1), st));
    int rc = check_data(s, d_data);
    if (rc) return rc;
    rc = single_level(s, (unsigned char *)d_data, n, 2, 0, 0, shift, bits, nullptr, st);
    if (rc) return rc;
    // the single segment's SegArrays start the state arena: bucket_begin first
    return cuda_status(cudaMemcpyAsync(d_bucket_begin, s.d_sarr, sizeof(uint64_t) * (B + 1),
                                       cudaMemcpyDeviceToDevice, st));
}

static int check_segmented(ipsgpu_sorter *h, void *d_data, uint64_t n, const uint64_t *d_offsets,
                           uint64_t nseg) {
    if (!h) return IPSGPU_E_INVAL;
    if (n > (1ull << 40) || nseg > 0xFFFFFFFFull) return IPSGPU_E_INVAL;
    if (nseg > 0 && (!d_offsets || ((uintptr_t)d_offsets % 8))) return IPSGPU_E_INVAL;
    if (n > 0 && nseg > 0) return check_data(h->s, d_data);
    return IPSGPU_OK;
}

int ipsgpu_sort_segmented(ipsgpu_sorter *h, void *d_data, uint64_t n, const uint64_t *d_offsets,
                          uint64_t num_segments, void *stream) {
    NvtxRange nvtx_range("ipsgpu_sort_segmented");
    int rc = check_segmented(h, d_data, n, d_offsets, num_segments);
    if (rc) return rc;
    if (n < 2 || num_segments == 0) return IPSGPU_OK;
    h->s.level_elems = n;
    return graph_run(h->s, make_job((unsigned char *)d_data, n, d_offsets, nullptr, num_segments,
                                    nullptr),
                     (cudaStream_t)stream);
}

int ipsgpu_sort_batch(ipsgpu_sorter *h, const uint64_t *d_segs, uint64_t num_segments,
                      void *stream) {
    NvtxRange nvtx_range("ipsgpu_sort_batch");
    if (!h || num_segments > 0xFFFFFFFFull) return IPSGPU_E_INVAL;
    if (num_segments == 0) return IPSGPU_OK;
    if (!d_segs || ((uintptr_t)d_segs % 8)) return IPSGPU_E_INVAL;
    h->s.level_elems = 0;
    return graph_run(h->s, make_job(nullptr, 0, nullptr, d_segs, num_segments, nullptr),
                     (cudaStream_t)stream);
}

struct ipsgpu_graph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

int ipsgpu_segmented_graph_create(ipsgpu_sorter *h, void *d_data, uint64_t n,
                                  const uint64_t *d_offsets, uint64_t num_segments,
                                  ipsgpu_graph **out) {
    NvtxRange nvtx_range("ipsgpu_segmented_graph_create");
    if (!out) return IPSGPU_E_INVAL;
    *out = nullptr;
    int rc = check_segmented(h, d_data, n, d_offsets, num_segments);
    if (rc) return rc;
    ipsgpu_graph *g = new (std::nothrow) ipsgpu_graph;
    if (!g) return IPSGPU_E_NOMEM;
    const GJob job = make_job((unsigned char *)d_data, n, d_offsets, nullptr, num_segments, nullptr);
    rc = build_wave_graph(h->s, &job, &g->graph, &g->exec);
    if (rc) {
        delete g;
        return rc;
    }
    *out = g;
    return IPSGPU_OK;
}

int ipsgpu_graph_launch(ipsgpu_graph *g, void *stream) {
    NvtxRange nvtx_range("ipsgpu_graph_launch");
    if (!g || !g->exec) return IPSGPU_E_INVAL;
    return cuda_status(cudaGraphLaunch(g->exec, (cudaStream_t)stream));
}

int ipsgpu_graph_nodes(ipsgpu_graph *g, uint64_t *nodes) {
    if (!g || !g->graph || !nodes) return IPSGPU_E_INVAL;
    size_t cnt = 0;
    if (cudaGraphGetNodes(g->graph, nullptr, &cnt) != cudaSuccess) return IPSGPU_E_CUDA;
    *nodes = cnt;
    return IPSGPU_OK;
}

int ipsgpu_graph_destroy(ipsgpu_graph *g) {
    if (!g) return IPSGPU_E_INVAL;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
    return IPSGPU_OK;
}

int ipsgpu_classify(ipsgpu_sorter *h, const void *d_data, uint64_t n, const void *d_splitters,
                    uint32_t num_splitters, int equal_buckets, uint32_t *d_class, void *stream) {
    NvtxRange nvtx_range("ipsgpu_classify");
    if (!h || !d_class || !d_splitters || num_splitters == 0) return IPSGPU_E_INVAL;
    Sorter &s = h->s;
    const uint64_t K = next_pow2((uint64_t)num_splitters + 1);
    const uint64_t B = equal_buckets ? 2 * K : K;
    if (B > s.k) return IPSGPU_E_INVAL;
    if (n == 0) return IPSGPU_OK;
    int rc = check_data(s, d_data);
    if (rc || (rc = check_data(s, d_splitters))) return rc;
    if ((rc = wait_uploads(s))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    s.data = (unsigned char *)d_data;
    SegDesc &sd = s.h_seg[0];
    memset(&sd, 0, sizeof sd);
    sd.addr = (uint64_t)(uintptr_t)d_data;
    sd.n = n;
    sd.b = s.b;
    sd.C = (uint32_t)B;
    sd.mode = 1;
    sd.nsplit = num_splitters;
    sd.eq_given = equal_buckets ? 1 : 0;
    BatchPlan bp;
    bp.nseg = 1;
    if ((rc = upload_plan(s, bp, st))) return rc;
    s.level_elems = n;
    const LevelArgs a = s.args(1, 0, 0, (uint32_t)B, (const unsigned char *)d_splitters);
    return cuda_status(s.ops->classify_ids(&s, a, d_class, st));
}

int ipsgpu_status(ipsgpu_sorter *h, void *stream) {
    if (!h) return IPSGPU_E_INVAL;
    Sorter &s = h->s;
    cudaStream_t st = (cudaStream_t)stream;
    int code = 0;
    int rc = read_status(s, st, &code);
    if (rc) return rc;
    if (cudaMemsetAsync(s.d_status, 0, sizeof(int), st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return IPSGPU_E_CUDA;
    return code;
}

const char *ipsgpu_strerror(int code) {
    switch (code) {
    case IPSGPU_OK: return "ok";
    case IPSGPU_E_INVAL: return "invalid argument";
    case IPSGPU_E_UNSUPPORTED: return "unsupported element type / algorithm combination";
    case IPSGPU_E_NOMEM: return "out of memory";
    case IPSGPU_E_CUDA: return "CUDA runtime error";
    case IPSGPU_E_TIMEOUT: return "a bounded device wait timed out";
    case IPSGPU_E_BUSY: return "request cannot be admitted now";
    case IPSGPU_E_INTERNAL: return "internal consistency check failed";
    case IPSGPU_E_CANCELED: return "request cancelled before it ran";
    default: return "unknown status";
    }
}

int ipsgpu_set_timing(ipsgpu_sorter *h, int enable) {
    if (!h) return IPSGPU_E_INVAL;
    h->s.timing = enable != 0;
    return IPSGPU_OK;
}

static const char *kKindNames[KK_COUNT] = {"detect", "reverse", "sample_tree", "classify",
                                           "prep",   "fixup",   "permute",     "stage",
                                           "fill",   "base_case", "classify_ids", "debug_wait",
                                           "plan"};

const char *ipsgpu_kernel_name(int kind) {
    return (kind >= 0 && kind < KK_COUNT) ? kKindNames[kind] : "";
}

int ipsgpu_kernel_stats(ipsgpu_sorter *h, uint64_t *launches, double *ms, double *bytes, int cap) {
    if (!h) return -IPSGPU_E_INVAL;
    Sorter &s = h->s;
    s.collect();
    for (int i = 0; i < KK_COUNT && i < cap; i++) {
        if (launches) launches[i] = s.stat_launches[i];
        if (ms) ms[i] = s.stat_ms[i];
        if (bytes) bytes[i] = s.stat_bytes[i];
        s.stat_launches[i] = 0;
        s.stat_ms[i] = 0;
        s.stat_bytes[i] = 0;
    }
    return KK_COUNT;
}

int ipsgpu_wave_stats(ipsgpu_sorter *h, uint64_t *waves, uint64_t *max_pending,
                      uint64_t *ring_capacity) {
    if (!h) return IPSGPU_E_INVAL;
    if (waves) *waves = h->s.last_waves;
    if (max_pending) *max_pending = h->s.last_max_pending;
    if (ring_capacity) *ring_capacity = h->s.ring_cap;
    return IPSGPU_OK;
}

int ipsgpu_debug_bounded_wait(ipsgpu_sorter *h, uint32_t spin_limit, void *stream) {
    if (!h) return IPSGPU_E_INVAL;
    Sorter &s = h->s;
    cudaStream_t st = (cudaStream_t)stream;
    s.tbegin(KK_WAIT, 0, st);
    k_debug_wait<<<1, 32, 0, st>>>(s.d_waitflag, spin_limit, s.d_status);
    s.tend(st);
    return cuda_status(cudaGetLastError());
}

}  // extern "C"

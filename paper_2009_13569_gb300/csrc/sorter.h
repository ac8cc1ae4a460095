// sorter.h -- host-side state of an ipsgpu_sorter and the per-element-type
// launch table.  Internal to the library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <nvtx3/nvToolsExt.h>

#include <vector>

#include "common.cuh"

namespace ipsgpu {

enum KernelKind {
    KK_DETECT = 0,
    KK_REVERSE,
    KK_SAMPLE,
    KK_CLASSIFY,
    KK_PREP,
    KK_FIXUP,
    KK_PERMUTE,
    KK_STAGE,
    KK_FILL,
    KK_BASE,
    KK_CLASSIFY_IDS,
    KK_WAIT,
    KK_PLAN,
    KK_COUNT
};

struct Sorter;
struct GraphArgs;

// Grid of each level kernel (work items are looped over, so any grid is
// correct; the host planner passes the exact counts).
struct LevelGrids {
    uint32_t seg, stripe, cta, cls;
};

// Kernel launchers of one element type (implemented in ops_<type>.cu).
struct TypeOps {
    int D;         // element bytes
    int key_bytes; // sizeof(K)
    cudaError_t (*init)(Sorter *);  // kernel attributes (idempotent)
    size_t (*classify_smem_bytes)(uint32_t k, uint32_t b);  // shared memory of k_classify
    cudaError_t (*level)(Sorter *, const LevelArgs &, const LevelGrids &, cudaStream_t);
    cudaError_t (*base)(Sorter *, const uint64_t *d_segs, uint32_t nsegs,
                        const uint32_t *nsegs_dev, uint32_t grid, cudaStream_t);
    cudaError_t (*detect)(Sorter *, const unsigned char *data, uint64_t n,
                          unsigned long long *mm, cudaStream_t);
    cudaError_t (*reverse)(Sorter *, unsigned char *data, uint64_t n, cudaStream_t);
    cudaError_t (*classify_ids)(Sorter *, const LevelArgs &, uint32_t *out, cudaStream_t);
    cudaError_t (*wave)(Sorter *, const GraphArgs &, cudaStream_t, int in_graph,
                        cudaGraphConditionalHandle);
};

extern const TypeOps ops_u32, ops_u64, ops_f64, ops_pair, ops_rec100, ops_quartet;

struct TimedLaunch {
    int kind;
    double bytes;
    cudaEvent_t ev0, ev1;
};

// NVTX range over a host-side call, so that profilers show which library
// call issued which kernels (no cost without an attached tool).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

constexpr uint64_t kGuardBytes = 256;
constexpr unsigned char kGuardByte = 0xA5;

struct Sorter {
    int dtype = 0;
    int device = 0;
    int nsm = 0;
    uint32_t perm_ctas = 0;  // k_permute CTAs resident at once on the device (set by ops->init)
    const TypeOps *ops = nullptr;
    // parameters (defaults resolved)
    uint32_t k = 256;
    uint32_t block_bytes = 512;
    float alpha_scale = 0.2f;
    uint64_t seed = 0;
    int algo = 0;
    uint32_t spin_limit = 1u << 22;
    uint64_t arena_bytes = 256ull << 20;
    uint32_t b = 64;        // block size in elements
    uint32_t smax = 24576;  // largest segment of the base case
    // capacities of one level (device-planned) or one host-planned batch
    uint32_t seg_cap = 1u << 16;     // segments
    uint32_t stripe_cap = 1u << 16;  // classification stripes
    uint32_t cta_cap = 1u << 17;     // block-permutation CTAs
    uint32_t cls_cap = 1u << 20;     // (segment, class) pairs
    uint32_t cnt_cap = 1u << 21;     // per-stripe class counters
    uint32_t move_cap = 1u << 22;    // fix-up moves
    uint32_t base_cap = 1u << 21;    // base-case segments per wave (>= cls_cap + feed)
    uint32_t ring_cap = 1u << 20;    // segments waiting for a partitioning step
    uint64_t sarr_bytes = 0, keys_bytes = 0;
    // device scratch
    SegDesc *d_seg = nullptr;
    SegState *d_st = nullptr;
    unsigned char *d_sarr = nullptr, *d_keys = nullptr;
    StripeDesc *d_stripe = nullptr;
    uint32_t *d_scount = nullptr, *d_sfull = nullptr;
    unsigned char *d_arena = nullptr;
    Move *d_moves = nullptr;
    uint32_t *d_nmoves = nullptr;
    int *d_status = nullptr;
    uint32_t *d_cta_seg = nullptr;
    uint64_t *d_base = nullptr;
    int *d_flags = nullptr;
    uint32_t *d_waitflag = nullptr;
    unsigned char *d_ring = nullptr;   // device planner: segments waiting (GList)
    uint32_t *d_stripe_first = nullptr;  // device planner: first stripe of each part
    unsigned char *d_gjob = nullptr;   // GJob of the current run
    unsigned char *d_gstate = nullptr; // GState of the current run
    unsigned char *h_gstate = nullptr; // pinned: GState read back by the host-driven loop
    cudaStream_t cap_stream = nullptr; // stream used to capture the wave graph
    cudaGraph_t wave_graph = nullptr;  // WHILE loop over waves (built on first use)
    cudaGraphExec_t wave_exec = nullptr;
    // pinned host mirrors
    SegDesc *h_seg = nullptr;
    StripeDesc *h_stripe = nullptr;
    uint32_t *h_cta_seg = nullptr;
    int *h_flags = nullptr;
    uint64_t scratch_bytes = 0;
    // Every device buffer sits between two guard zones of kGuardBytes filled
    // with kGuardByte at creation; a kernel writing past either end of its
    // buffer changes a guard (ipsgpu_debug_check_guards).
    struct Guarded {
        unsigned char *base;  // the allocation: guard | buffer | guard
        uint64_t bytes;       // the buffer
    };
    std::vector<Guarded> guarded;
    cudaEvent_t h2d_done = nullptr;  // last upload out of the pinned mirrors
    // the level currently being launched
    unsigned char *data = nullptr;
    // timing
    bool timing = false;
    std::vector<TimedLaunch> launches;
    std::vector<cudaEvent_t> event_pool;
    uint64_t stat_launches[KK_COUNT] = {};
    double stat_ms[KK_COUNT] = {};
    double stat_bytes[KK_COUNT] = {};
    // per-level algorithmic element count (for the byte model of a launch)
    uint64_t level_elems = 0;
    // waves and peak ring occupancy of the last host-driven run
    uint64_t last_waves = 0, last_max_pending = 0;

    void tbegin(int kind, double bytes, cudaStream_t st);
    void tend(cudaStream_t st);
    void collect();
    LevelArgs args(uint32_t nseg, uint32_t nstripe, uint32_t ncta, uint32_t ncls,
                   const unsigned char *given_spl) const;
};

}  // namespace ipsgpu

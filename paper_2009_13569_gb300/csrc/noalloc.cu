// noalloc.cu -- ipsgpu_partition_level_noalloc: one partitioning level with
// given splitters that allocates no memory.
//
// Some callers cannot call cudaMalloc: code that runs while a CUDA graph is
// being captured, code inside an allocator or a memory-pool callback, or a
// service that reserves all device memory up front and forbids later
// allocations.  A sorter (ipsgpu_sorter_create) allocates its scratch, so
// those callers cannot create one.  This entry point keeps its scratch in a
// fixed, file-scope device array instead, so every call runs with memory
// that was reserved when the library was loaded.
//
// The array holds one segment's state, at most kNaStripes stripes with their
// leftover buffer blocks, and the fix-up and permutation bookkeeping:
// kNaScratchBytes in total (about 8.2 MiB), present on every GPU that loads
// the library until the process exits.  Its device address is obtained once
// per device with cudaGetSymbolAddress on the first call made with that
// device current (a host-side name of a __device__ array is not a device
// address).  That first call also sets the kernel attributes of every
// element type, so it should not be made while a stream is being captured.
//
// All calls share the array and each leaves its contents behind; the parts
// that must start at zero (move counter, status word) are cleared by every
// call.  Two calls whose work overlaps on the GPU (different streams, or
// different host threads) therefore race and must be serialized by the
// caller.
#include <string.h>

#include <mutex>

#include "sorter.h"

using namespace ipsgpu;

namespace {

constexpr uint32_t kNaStripes = 64;
constexpr uint32_t kNaCtas = 2048;
constexpr uint32_t kNaMoves = 2 * (kNaStripes + kMaxClasses) + 4;
constexpr uint64_t kNaSlot = (uint64_t)kMaxClasses * 512;  // leftover buffers of one stripe
constexpr uint64_t kNaMaxN = 0xFFFFFFFFull;                // elements per call
constexpr int kNaMaxDevices = 64;
constexpr int kNaTypes = IPSGPU_QUARTET + 1;

constexpr uint64_t al(uint64_t x) { return (x + 255) & ~(uint64_t)255; }
// cleanup staging of C <= 256 blocks of <= 512 bytes, then the overflow block
constexpr uint64_t kNaStage = al(kNaSlot + 512);
constexpr uint64_t kOSeg = 0;
constexpr uint64_t kOSt = al(kOSeg + sizeof(SegDesc));
constexpr uint64_t kOSarr = al(kOSt + sizeof(SegState));   // SegArrays: bucket_begin first
constexpr uint64_t kOKeys = al(kOSarr + 28 * kMaxClasses + 32);  // tree, splitters
constexpr uint64_t kOStripe = al(kOKeys + 2 * kMaxClasses * sizeof(Key192));  // widest key
constexpr uint64_t kOScount = al(kOStripe + kNaStripes * sizeof(StripeDesc));
constexpr uint64_t kOSfull = al(kOScount + (uint64_t)kNaStripes * kMaxClasses * 4);
constexpr uint64_t kOMoves = al(kOSfull + kNaStripes * 4);
constexpr uint64_t kONmoves = al(kOMoves + kNaMoves * sizeof(Move));
constexpr uint64_t kOStatus = kONmoves + 4;
constexpr uint64_t kOCta = al(kOStatus + 4);
constexpr uint64_t kOArena = al(kOCta + kNaCtas * 4);
constexpr uint64_t kNaScratchBytes = kOArena + kNaStage + kNaStripes * kNaSlot;

static __device__ __align__(256) unsigned char g_na_scratch[kNaScratchBytes];

struct DeviceSetup {
    std::mutex mu;
    bool done[kNaMaxDevices] = {};
    unsigned char *ptr[kNaMaxDevices] = {};
    int nsm[kNaMaxDevices] = {};
};
DeviceSetup g_setup;

// Descriptors of the single segment, its stripes and its permutation CTAs,
// written on the device from scalar arguments (no host upload).
__global__ void k_na_plan(unsigned char *scr, uint64_t addr, uint64_t n, uint32_t b, uint32_t C,
                          uint32_t p,
                          uint32_t nc, uint32_t nsplit, uint32_t eq, uint32_t slot_bytes) {
    SegDesc *sd = reinterpret_cast<SegDesc *>(scr + kOSeg);
    StripeDesc *sp = reinterpret_cast<StripeDesc *>(scr + kOStripe);
    uint32_t *cta = reinterpret_cast<uint32_t *>(scr + kOCta);
    const uint64_t nb = (n + b - 1) / b;
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t == 0) {
        SegDesc d;
        memset(&d, 0, sizeof d);
        d.addr = addr;
        d.n = n;
        d.b = b;
        d.C = C;
        d.stripe0 = 0;
        d.nstripes = p;
        d.cta0 = 0;
        d.ncta = nc;
        d.stage_off = 0;
        d.arr_off = 0;
        d.key_off = 0;
        d.cls0 = 0;
        d.cnt0 = 0;
        d.mode = 1;
        d.nsplit = nsplit;
        d.eq_given = eq;
        *sd = d;
        *reinterpret_cast<uint32_t *>(scr + kONmoves) = 0;
        *reinterpret_cast<int *>(scr + kOStatus) = 0;
    }
    if (t < p) {
        StripeDesc q;
        q.seg = 0;
        q.blk0 = (uint32_t)(t * nb / p);
        q.nblk = (uint32_t)((t + 1) * nb / p - t * nb / p);
        q.cnt_off = t * C;
        q.left_off = kNaStage + (uint64_t)t * slot_bytes;
        sp[t] = q;
    }
    if (t < nc) cta[t] = 0;
}

// bucket_begin[0..B] to the caller; an error seen by any kernel of this call
// turns the total bucket_begin[B] into ~0 so the caller can detect it
__global__ void k_na_finish(const unsigned char *scr, uint64_t *out, uint32_t B) {
    const uint64_t *bb = reinterpret_cast<const uint64_t *>(scr + kOSarr);
    const int status = *reinterpret_cast<const int *>(scr + kOStatus);
    for (uint32_t j = threadIdx.x; j <= B; j += blockDim.x)
        out[j] = (j == B && status != 0) ? ~0ull : bb[j];
}

const TypeOps *na_ops(int dtype) {
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

}  // namespace

extern "C" int ipsgpu_partition_level_noalloc(int dtype, void *d_data, uint64_t n,
                                              const void *d_splitters, uint32_t num_splitters,
                                              int equal_buckets, uint64_t *d_bucket_begin,
                                              void *stream) {
    const TypeOps *ops = na_ops(dtype);
    if (!ops || !d_bucket_begin || !d_splitters || num_splitters == 0) return IPSGPU_E_INVAL;
    uint64_t K = 1;
    while (K < (uint64_t)num_splitters + 1) K <<= 1;
    const uint64_t B = equal_buckets ? 2 * K : K;
    if (B > kMaxClasses || n > kNaMaxN) return IPSGPU_E_INVAL;
    cudaStream_t st = (cudaStream_t)stream;
    if (n == 0)
        return cudaMemsetAsync(d_bucket_begin, 0, sizeof(uint64_t) * (B + 1), st) == cudaSuccess
                   ? IPSGPU_OK
                   : IPSGPU_E_CUDA;
    const uintptr_t al_req = ops->D == 100 ? 4 : (uintptr_t)(ops->D < 16 ? ops->D : 16);
    if (!d_data || ((uintptr_t)d_data % al_req) || ((uintptr_t)d_splitters % al_req))
        return IPSGPU_E_INVAL;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices) return IPSGPU_E_CUDA;
    Sorter s;  // a view onto the static array: no member allocates
    s.dtype = dtype;
    s.ops = ops;
    uint32_t b = 1;
    while ((uint64_t)b * 2 * ops->D <= 512) b *= 2;
    s.b = b;
    {
        std::lock_guard<std::mutex> lock(g_setup.mu);
        if (!g_setup.done[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_na_scratch) != cudaSuccess || !p) return IPSGPU_E_CUDA;
            int nsm = 0;
            if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
                return IPSGPU_E_CUDA;
            // kernel attributes of every element type now, so that no later
            // call (of another dtype) sets any
            for (int t = 0; t < kNaTypes; t++)
                if (na_ops(t)->init(&s) != cudaSuccess) return IPSGPU_E_CUDA;
            g_setup.ptr[dev] = static_cast<unsigned char *>(p);
            g_setup.nsm[dev] = nsm;
            g_setup.done[dev] = true;
        }
    }
    unsigned char *scr = g_setup.ptr[dev];
    const int nsm = g_setup.nsm[dev];
    s.nsm = nsm;
    s.k = kMaxClasses;
    s.d_seg = reinterpret_cast<SegDesc *>(scr + kOSeg);
    s.d_st = reinterpret_cast<SegState *>(scr + kOSt);
    s.d_sarr = scr + kOSarr;
    s.d_keys = scr + kOKeys;
    s.d_stripe = reinterpret_cast<StripeDesc *>(scr + kOStripe);
    s.d_scount = reinterpret_cast<uint32_t *>(scr + kOScount);
    s.d_sfull = reinterpret_cast<uint32_t *>(scr + kOSfull);
    s.d_arena = scr + kOArena;
    s.d_moves = reinterpret_cast<Move *>(scr + kOMoves);
    s.d_nmoves = reinterpret_cast<uint32_t *>(scr + kONmoves);
    s.d_status = reinterpret_cast<int *>(scr + kOStatus);
    s.d_cta_seg = reinterpret_cast<uint32_t *>(scr + kOCta);
    s.move_cap = kNaMoves;
    s.data = static_cast<unsigned char *>(d_data);
    s.level_elems = n;

    // the same stripe and CTA sizing as a sorter, clamped to the array
    const uint64_t nb = (n + b - 1) / b;
    uint64_t stripe_elems = n / (2 * (uint64_t)nsm);
    if (stripe_elems < (1u << 15)) stripe_elems = 1u << 15;
    uint64_t p = (n + stripe_elems - 1) / stripe_elems;
    if (p > kNaStripes) p = kNaStripes;
    if (p > nb) p = nb;
    if (p < 1) p = 1;
    uint64_t bpc = nb / (8 * (uint64_t)nsm);
    if (bpc < 32) bpc = 32;
    uint64_t nc = (nb + bpc - 1) / bpc;
    if (nc > kNaCtas) nc = kNaCtas;
    if (nc < 1) nc = 1;
    const uint32_t threads = 256;
    const uint32_t work = (uint32_t)(p > nc ? p : nc);
    k_na_plan<<<(work + threads - 1) / threads, threads, 0, st>>>(
        scr, (uint64_t)(uintptr_t)d_data, n, b, (uint32_t)B, (uint32_t)p, (uint32_t)nc,
        num_splitters, equal_buckets ? 1u : 0u, (uint32_t)kNaSlot);
    if (cudaGetLastError() != cudaSuccess) return IPSGPU_E_CUDA;
    const LevelArgs a = s.args(1, (uint32_t)p, (uint32_t)nc, (uint32_t)B,
                               static_cast<const unsigned char *>(d_splitters));
    const LevelGrids g{1, (uint32_t)p, (uint32_t)nc, (uint32_t)B};
    if (ops->level(&s, a, g, st) != cudaSuccess) return IPSGPU_E_CUDA;
    k_na_finish<<<1, 256, 0, st>>>(scr, d_bucket_begin, (uint32_t)B);
    return cudaGetLastError() == cudaSuccess ? IPSGPU_OK : IPSGPU_E_CUDA;
}

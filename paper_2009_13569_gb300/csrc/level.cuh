// level.cuh -- kernels of one in-place partitioning step over a batch of
// segments (Sec. 3.1 of Axtmann et al.):
//   k_sample_tree  sampling, splitter selection, dedupe, branchless tree
//                  (Sec. 3.1.1, Sec. 2)
//   k_classify     classification into per-bucket buffer blocks, full blocks
//                  flushed to the front of the stripe (Sec. 3.1.2;
//                  classify.cuh)
//   k_prep         bucket sizes -> prefix sum -> delimiters, per-bucket
//                  (write, read) pointers, stripe-boundary fix-up plan
//                  (Sec. 3.1.3, first part)
//   k_fixup        moves full blocks into the empty slots of their bucket
//                  region so every region is (full blocks | empty blocks)
//   k_permute      the block permutation with atomic (w, r) pointer pairs,
//                  reader counts and two swap buffers per worker
//                  (Sec. 3.1.3)
//   k_stage/k_fill cleanup of bucket heads and tails from the overflowing
//                  last block, the leftover buffer blocks and the overflow
//                  block (Sec. 3.1.4)
// Every kernel loops over its work items (segments, stripes, CTAs or
// (segment, class) pairs), so the same kernels serve a host-planned batch
// and a device-planned one whose counts live in device memory.
#pragma once

#include "common.cuh"

namespace ipsgpu {

constexpr int kSampleThreads = 1024;
// Samples per bucket: bucket sizes spread by about 1/sqrt of it, and every
// child above the base-case size costs another partitioning pass, so the
// sample is larger than the paper's alpha k on the GPU.
constexpr uint32_t kMinSamplesPerBucket = 64;
constexpr int kPermuteThreads = 256;
constexpr int kAuxThreads = 256;

template <class T>
struct LevelClassifier {
    typedef typename T::K K;
    typedef typename T::E E;
    const K *tree;
    const K *spl;
    uint32_t logK;
    bool eq;
    bool radix;
    uint32_t shift;
    uint64_t mask;
    __device__ __forceinline__ uint32_t operator()(const E &e) const {
        if (radix) return (uint32_t)((T::rkey(e) >> shift) & mask);
        return classify_key<K>(T::key(e), tree, spl, logK, eq);
    }
    // The same class computed by a whole warp (every lane passes the same
    // element and gets the class), in two vote steps instead of logK
    // dependent tree steps.  The class index is the number of padded
    // splitters s_0..s_{K-2} below the key.  For K <= 32 those are exactly
    // the tree nodes 1..K-1; for K > 32 the tree's top nodes 1..31 are the
    // splitters s_{S m - 1} (m = 1..31, S = K / 32) that close each group of
    // S consecutive splitters, so the first vote counts the groups entirely
    // below the key and the second counts inside the next group.
    __device__ __forceinline__ uint32_t warp_class(const E &e, int lane) const {
        if (radix) return (uint32_t)((T::rkey(e) >> shift) & mask);
        const K k = T::key(e);
        const uint32_t nk = 1u << logK;
        uint32_t i;
        if (nk <= 32) {
            const bool below = lane >= 1 && (uint32_t)lane < nk && tree[lane] < k;
            i = __popc(__ballot_sync(0xffffffffu, below));
        } else {
            const uint32_t S = nk >> 5;
            const bool below = lane >= 1 && tree[lane] < k;
            const uint32_t q = __popc(__ballot_sync(0xffffffffu, below));
            const uint32_t j = q * S + (uint32_t)lane;
            const bool below2 = (uint32_t)lane < S && j < nk - 1 && spl[j] < k;
            i = q * S + __popc(__ballot_sync(0xffffffffu, below2));
        }
        if (eq) i = 2 * i + 1 - (k < spl[i] ? 1u : 0u);
        return i;
    }
};

template <class T>
__device__ __forceinline__ const typename T::K *seg_tree(const LevelArgs &a, const SegDesc &sd) {
    return reinterpret_cast<const typename T::K *>(a.keys + sd.key_off);
}
template <class T>
__device__ __forceinline__ const typename T::K *seg_spl(const LevelArgs &a, const SegDesc &sd) {
    return reinterpret_cast<const typename T::K *>(a.keys + sd.key_off) + sd.C;
}

// Copies the segment's splitters, and its tree unless s_tree is null, into
// shared memory; callers sync.
template <class T>
__device__ __forceinline__ void load_classifier(LevelClassifier<T> &c, const LevelArgs &a,
                                                const SegDesc &sd, const SegState &st,
                                                typename T::K *s_tree, typename T::K *s_spl) {
    typedef typename T::K K;
    c.radix = sd.mode == 2;
    c.shift = sd.radix_shift;
    c.mask = (sd.radix_bits >= 64) ? ~0ull : ((1ull << sd.radix_bits) - 1);
    c.logK = st.logK;
    c.eq = st.eq != 0;
    c.tree = s_tree;
    c.spl = s_spl;
    if (!c.radix) {
        const K *gt = seg_tree<T>(a, sd);
        const K *gs = seg_spl<T>(a, sd);
        for (uint32_t i = threadIdx.x; i < st.K; i += blockDim.x) {
            if (s_tree) s_tree[i] = gt[i];
            s_spl[i] = gs[i];
        }
    }
}

// ------------------------------------------------------------------- K1
// One CTA per segment.  mode 0: sample, sort the sample in shared memory,
// pick equidistant splitters, remove duplicates; if duplicates existed, use
// equality buckets with half as many leaves so the class count stays within
// the budget C.  mode 1: splitters given.  mode 2: radix digits.
// Then pad to K = 2^ceil(log2(m+1)) and lay out the BFS tree.
template <class T>
__global__ void __launch_bounds__(kSampleThreads) k_sample_tree(LevelArgs a) {
    typedef typename T::K K;
    typedef typename T::E E;
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr uint32_t kMaxSample = max_sort_sample<K>();
    K *smp = reinterpret_cast<K *>(smem);                       // kMaxSample
    K *cand = smp + kMaxSample;                                 // kMaxClasses
    uint32_t *flag = reinterpret_cast<uint32_t *>(cand + kMaxClasses);  // kMaxClasses
    uint32_t *pos = flag + kMaxClasses;                         // kMaxClasses
    uint32_t *wtmp = pos + kMaxClasses;                         // 34
    __shared__ uint32_t sh_eq, sh_d;
    const int tid = threadIdx.x;
    const uint32_t nseg = lv_nseg(a);

    for (uint32_t s = blockIdx.x; s < nseg; s += gridDim.x) {
        const SegDesc sd = a.seg[s];
        SegState *st = a.st + s;
        const uint32_t b = sd.b;
        if (tid == 0) {
            st->nslots = (uint32_t)((sd.n + b - 1) / b);
            st->nfull_slots = (uint32_t)(sd.n / b);
            st->ovf_used = 0;
        }
        if (sd.mode == 2) {
            if (tid == 0) {
                st->K = 1u << sd.radix_bits;
                st->B = 1u << sd.radix_bits;
                st->logK = sd.radix_bits;
                st->eq = 0;
            }
            continue;
        }
        K *gtree = reinterpret_cast<K *>(a.keys + sd.key_off);
        K *gspl = gtree + sd.C;
        const E *base = reinterpret_cast<const E *>(sd.addr);

        if (sd.mode == 1) {
            const E *g = reinterpret_cast<const E *>(a.given_spl);
            for (uint32_t j = tid; j < sd.nsplit; j += blockDim.x) cand[j] = T::key(g[j]);
            if (tid == 0) {
                sh_d = sd.nsplit;
                sh_eq = sd.eq_given;
            }
            __syncthreads();
        } else {
            // sample size: alpha * C, alpha = max(1, alpha_scale * log2 n)
            // (Sec. 5), raised to at least kMinSamplesPerBucket per bucket
            // so that children stay within the base-case capacity, at most
            // what one CTA sorts
            const uint32_t C = sd.C;
            float alpha = a.alpha_scale * log2f((float)sd.n);
            if (alpha < 1.f) alpha = 1.f;
            uint32_t m = (uint32_t)(alpha * (float)C);
            if (m < kMinSamplesPerBucket * C) m = kMinSamplesPerBucket * C;
            if (m < C - 1) m = C - 1;
            if (m > kMaxSample) m = kMaxSample;
            uint32_t P = 1;
            while (P < m) P <<= 1;
            const uint64_t sseed = a.seed ^ (sd.addr * 0xD1B54A32D192ED03ull) ^ (sd.n << 17);
            // random gather, four keys in flight per thread
            for (uint32_t t0 = tid; t0 < P; t0 += 4 * blockDim.x) {
                K kx[4];
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const uint32_t t = t0 + q * blockDim.x;
                    if (t < m) {
                        const uint64_t idx = splitmix64(sseed + t * 0x9E3779B97F4A7C15ull) % sd.n;
                        kx[q] = T::key(base[idx]);
                    }
                }
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const uint32_t t = t0 + q * blockDim.x;
                    if (t < P) smp[t] = t < m ? kx[q] : T::max_key();
                }
            }
            __syncthreads();
            // bitonic sort of smp[0..P); j is a power of two, so compare-
            // exchange i pairs lo = 2 j (i / j) + i mod j with lo + j
            for (uint32_t k = 2; k <= P; k <<= 1) {
                for (uint32_t j = k >> 1, lj = ilog2_floor(k) - 1; j > 0; j >>= 1, lj--) {
                    for (uint32_t i = tid; i < P / 2; i += blockDim.x) {
                        const uint32_t lo = ((i >> lj) << (lj + 1)) | (i & (j - 1));
                        const uint32_t hi = lo + j;
                        bool up = (lo & k) == 0;
                        K x = smp[lo], y = smp[hi];
                        if ((y < x) == up) {
                            smp[lo] = y;
                            smp[hi] = x;
                        }
                    }
                    __syncthreads();
                }
            }
            // equidistant splitters, dedupe.  If any duplicate was found the
            // level uses equality buckets: the splitters are picked again for
            // C/2 leaves so that the 2K classes still fit the budget C.
            uint32_t Cc = C;
            for (int attempt = 0; attempt < 2; attempt++) {
                const uint32_t ns = Cc - 1;
                for (uint32_t j = tid; j < ns; j += blockDim.x)
                    cand[j] = smp[((uint64_t)(j + 1) * m) / Cc - 1];
                __syncthreads();
                for (uint32_t j = tid; j < ns; j += blockDim.x)
                    flag[j] = (j == 0 || cand[j - 1] < cand[j]) ? 1u : 0u;
                __syncthreads();
                uint32_t d = cta_exclusive_scan<uint32_t>(flag, pos, (int)ns, wtmp);
                K keep = T::max_key();
                bool mine = false;
                uint32_t mypos = 0;
                // ns <= 255 < blockDim.x: each thread holds at most one entry
                for (uint32_t j = tid; j < ns; j += blockDim.x) {
                    if (flag[j]) {
                        keep = cand[j];
                        mine = true;
                        mypos = pos[j];
                    }
                }
                __syncthreads();
                if (mine) cand[mypos] = keep;
                if (tid == 0) {
                    sh_d = d;
                    if (attempt == 0) sh_eq = (d < ns) ? 1u : 0u;
                }
                __syncthreads();
                if (sh_eq == 0 || attempt == 1 || Cc < 4) break;
                Cc >>= 1;
                __syncthreads();
            }
        }
        const uint32_t d = sh_d;
        const uint32_t eq = sh_eq;
        uint32_t K_ = 1;
        while (K_ < d + 1) K_ <<= 1;
        const uint32_t logK = ilog2_floor(K_);
        for (uint32_t j = tid; j < K_; j += blockDim.x) gspl[j] = cand[j < d ? j : d - 1];
        for (uint32_t i = tid; i < K_; i += blockDim.x) {
            if (i == 0) continue;
            uint32_t l = ilog2_floor(i);
            uint32_t q = i - (1u << l);
            uint32_t idx = (2 * q + 1) * (K_ >> (l + 1)) - 1;
            gtree[i] = cand[idx < d ? idx : d - 1];
        }
        if (tid == 0) {
            st->K = K_;
            st->logK = logK;
            st->eq = eq;
            st->B = eq ? 2 * K_ : K_;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------- prep
// One CTA per segment: bucket sizes, prefix sum, delimiters rounded up to a
// block, per-bucket (w, r) pointers and the fix-up moves that make every
// bucket region "full blocks, then empty blocks" (Sec. 3.1.3).
__device__ inline uint32_t first_stripe_ending_after(const StripeDesc *sp, uint32_t s0,
                                                     uint32_t ns, uint32_t x) {
    // smallest stripe index i in [s0, s0+ns) with blk0 + nblk > x
    uint32_t lo = s0, hi = s0 + ns;
    while (lo < hi) {
        uint32_t mid = (lo + hi) >> 1;
        if (sp[mid].blk0 + sp[mid].nblk > x)
            hi = mid;
        else
            lo = mid + 1;
    }
    return lo;
}

struct RunIter {
    // iterates maximal runs of full (want_full) or empty slots in [x, y)
    const StripeDesc *sp;
    const uint32_t *sfull;
    uint32_t s, s_end, x, y;
    bool want_full;
    __device__ bool next(uint32_t &rs, uint32_t &re) {
        while (s < s_end && x < y) {
            const StripeDesc &d = sp[s];
            uint32_t fb = d.blk0 + sfull[s];   // end of the stripe's full part
            uint32_t se = d.blk0 + d.nblk;
            uint32_t lo = want_full ? d.blk0 : fb;
            uint32_t hi = want_full ? fb : se;
            lo = max(lo, x);
            hi = min(hi, min(se, y));
            if (x >= se) {
                s++;
                continue;
            }
            if (lo < hi) {
                rs = lo;
                re = hi;
                x = hi;
                if (x >= se) s++;
                return true;
            }
            x = se;
            s++;
        }
        return false;
    }
};

static __global__ void __launch_bounds__(kAuxThreads) k_prep(LevelArgs a) {
    __shared__ unsigned long long sz[kMaxClasses];
    __shared__ unsigned long long pre[kMaxClasses];
    __shared__ unsigned long long wtmp[34];
    const int tid = threadIdx.x;
    const uint32_t nseg = lv_nseg(a);
    for (uint32_t s = blockIdx.x; s < nseg; s += gridDim.x) {
        const SegDesc sd = a.seg[s];
        SegState *st = a.st + s;
        const SegArrays ar = seg_arrays(a.sarr, sd);
        const uint32_t B = st->B;
        const uint32_t b = sd.b;
        const uint32_t lb = ilog2_floor(b);
        const uint32_t nslots = st->nslots;
        for (uint32_t j = tid; j < B; j += blockDim.x) {
            unsigned long long sum = 0;
            uint32_t full = 0;
            for (uint32_t q = 0; q < sd.nstripes; q++) {
                uint32_t c = a.scount[a.stripe[sd.stripe0 + q].cnt_off + j];
                sum += c;
                full += c >> lb;
            }
            sz[j] = sum;
            ar.full[j] = full;
        }
        __syncthreads();
        const unsigned long long total = cta_exclusive_scan<unsigned long long>(sz, pre, (int)B, wtmp);
        if (total != sd.n) {
            // counts that do not add up to the segment (they would send
            // pointers past it): report, and leave the level nothing to move
            // (empty buckets, no blocks, no readers)
            if (tid == 0) set_status(a.status, IPSGPU_E_INTERNAL);
            for (uint32_t j = tid; j <= B; j += blockDim.x) {
                ar.bb[j] = 0;
                ar.dlm[j] = 0;
                if (j < B) {
                    ar.full[j] = 0;
                    ar.readers[j] = 0;
                    ar.ptr[j] = (unsigned long long)kRBias;
                }
            }
            __syncthreads();
            continue;
        }
        for (uint32_t j = tid; j <= B; j += blockDim.x) {
            uint64_t bb = j < B ? pre[j] : sd.n;
            ar.bb[j] = bb;
            ar.dlm[j] = j < B ? (uint32_t)((bb + b - 1) >> lb) : nslots;
        }
        __syncthreads();
        const StripeDesc *sp = a.stripe;
        for (uint32_t j = tid; j < B; j += blockDim.x) {
            const uint32_t lo = ar.dlm[j], hi = ar.dlm[j + 1];
            uint32_t f = 0;
            if (lo < hi) {
                RunIter it{sp, a.sfull, first_stripe_ending_after(sp, sd.stripe0, sd.nstripes, lo),
                           sd.stripe0 + sd.nstripes, lo, hi, true};
                uint32_t rs, re;
                while (it.next(rs, re)) f += re - rs;
            }
            ar.ptr[j] = ((unsigned long long)lo << 32) | (unsigned long long)(lo + f + kRBias);
            ar.readers[j] = 0;
            // fix-up: empty slots in [lo, lo+f) <- full slots in [lo+f, hi)
            const uint32_t P = lo + f;
            if (f > 0 && P < hi) {
                RunIter ei{sp, a.sfull, first_stripe_ending_after(sp, sd.stripe0, sd.nstripes, lo),
                           sd.stripe0 + sd.nstripes, lo, P, false};
                RunIter fi{sp, a.sfull, first_stripe_ending_after(sp, sd.stripe0, sd.nstripes, P),
                           sd.stripe0 + sd.nstripes, P, hi, true};
                uint32_t es = 0, ee = 0, fs = 0, fe = 0;
                while (true) {
                    if (es == ee && !ei.next(es, ee)) break;
                    if (fs == fe && !fi.next(fs, fe)) {
                        set_status(a.status, IPSGPU_E_INTERNAL);
                        break;
                    }
                    uint32_t len = min(ee - es, fe - fs);
                    uint32_t mi = atomicAdd(a.nmoves, 1u);
                    if (mi < a.move_cap) {
                        a.moves[mi] = Move{s, fs, es, len};
                    } else {
                        set_status(a.status, IPSGPU_E_INTERNAL);
                    }
                    es += len;
                    fs += len;
                }
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------ block copies
// A block of BB bytes (a multiple of 16, at most kMaxBlockBytes) is held by
// one warp in NV = ceil(BB / 512) 16-byte registers per lane: unit c of lane
// l holds bytes [512 c + 16 l, 512 c + 16 l + 16), so lane 0's unit 0 (and
// lane 1's for 32-byte elements) holds the first element.  `u` is the widest
// access unit (16, 8 or 4 bytes) both addresses allow.

template <int NV>
struct WarpBlock {
    uint4 v[NV];
};

template <int NV>
__device__ __forceinline__ void warp_load_block(WarpBlock<NV> &r, const unsigned char *p,
                                                uint32_t BB, int lane, int u) {
#pragma unroll
    for (int c = 0; c < NV; c++) {
        const uint32_t o = (uint32_t)c * 512 + (uint32_t)lane * 16;
        if (o >= BB) break;
        if (u == 16) {
            r.v[c] = __ldcg(reinterpret_cast<const uint4 *>(p + o));
        } else if (u == 8) {
            const uint2 *q = reinterpret_cast<const uint2 *>(p + o);
            uint2 x = __ldcg(q), y = __ldcg(q + 1);
            r.v[c] = make_uint4(x.x, x.y, y.x, y.y);
        } else {
            const uint32_t *q = reinterpret_cast<const uint32_t *>(p + o);
            r.v[c] = make_uint4(__ldcg(q), __ldcg(q + 1), __ldcg(q + 2), __ldcg(q + 3));
        }
    }
}

template <int NV>
__device__ __forceinline__ void warp_store_block(const WarpBlock<NV> &r, unsigned char *p,
                                                 uint32_t BB, int lane, int u) {
#pragma unroll
    for (int c = 0; c < NV; c++) {
        const uint32_t o = (uint32_t)c * 512 + (uint32_t)lane * 16;
        if (o >= BB) break;
        if (u == 16) {
            __stcg(reinterpret_cast<uint4 *>(p + o), r.v[c]);
        } else if (u == 8) {
            uint2 *q = reinterpret_cast<uint2 *>(p + o);
            __stcg(q, make_uint2(r.v[c].x, r.v[c].y));
            __stcg(q + 1, make_uint2(r.v[c].z, r.v[c].w));
        } else {
            uint32_t *q = reinterpret_cast<uint32_t *>(p + o);
            __stcg(q, r.v[c].x);
            __stcg(q + 1, r.v[c].y);
            __stcg(q + 2, r.v[c].z);
            __stcg(q + 3, r.v[c].w);
        }
    }
}

// 16-byte units per lane for blocks of BB bytes
__host__ __device__ inline int block_units(uint32_t BB) { return BB <= 512 ? 1 : (BB <= 1024 ? 2 : 4); }

__device__ __forceinline__ int access_unit(uint64_t byte_off) {
    return (byte_off & 15) == 0 ? 16 : ((byte_off & 7) == 0 ? 8 : 4);
}

// the segment's overflow block sits after its C staging blocks
__device__ __forceinline__ unsigned char *seg_ovf(const LevelArgs &a, const SegDesc &sd, int D) {
    return a.arena + sd.stage_off + (uint64_t)sd.C * sd.b * D;
}

// ------------------------------------------------------------------ fixup
template <class T, int NV>
__global__ void __launch_bounds__(kAuxThreads) k_fixup(LevelArgs a) {
    const uint32_t nm = min(*a.nmoves, a.move_cap);
    const int lane = threadIdx.x & 31;
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    // each warp walks the (move, block) pairs with a stride
    uint32_t m = 0, k = 0;
    uint32_t skip = gw;
    for (; m < nm; m++) {
        uint32_t len = a.moves[m].len;
        if (skip < len) {
            k = skip;
            break;
        }
        skip -= len;
    }
    while (m < nm) {
        const Move mv = a.moves[m];
        const SegDesc &sd = a.seg[mv.seg];
        const uint32_t BB = sd.b * T::D;
        unsigned char *base = reinterpret_cast<unsigned char *>(sd.addr);
        const int u = access_unit((uint64_t)(uintptr_t)base);
        WarpBlock<NV> r;
        warp_load_block<NV>(r, base + (uint64_t)(mv.src + k) * BB, BB, lane, u);
        warp_store_block<NV>(r, base + (uint64_t)(mv.dst + k) * BB, BB, lane, u);
        // advance by nwarps blocks
        uint32_t adv = nwarps;
        while (m < nm) {
            uint32_t len = a.moves[m].len;
            if (k + adv < len) {
                k += adv;
                break;
            }
            adv -= len - k;
            k = 0;
            m++;
        }
    }
}

// ---------------------------------------------------------------- permute
// Block permutation (Sec. 3.1.3).  Each warp is one worker with two swap
// buffers (one block per buffer, NV 16-byte registers per lane).  Per
// bucket i, ptr[i] packs the write pointer w_i (high half) and the exclusive
// read pointer r_i + 1 (low half, biased), so that one 64-bit atomic reads
// and modifies both consistently.  Blocks in [d_i, w_i) are correct, blocks
// in [w_i, r_i] unprocessed, the rest empty.  A CTA runs the virtual CTAs
// blockIdx.x, blockIdx.x + gridDim.x, ... of the level; workers of a segment
// never wait for one another except for the bounded reader wait, so they need
// not run at the same time.  The bucket of a block is that of its first
// element, classified by the whole warp (LevelClassifier::warp_class).
// One-unit blocks (up to 512 bytes) run six CTAs per SM (40 registers, a few
// spilled): the workers wait on global atomics and block loads, and more
// of them in flight beat the spills (2^30 uint64: 8.25 against 8.7 ms per
// sort at five CTAs per SM).
template <class T, int NV>
__global__ void __launch_bounds__(kPermuteThreads, NV == 1 ? 6 : 1) k_permute(LevelArgs a) {
    typedef typename T::K K;
    typedef typename T::E E;
    __shared__ K s_tree[kMaxClasses];
    __shared__ K s_spl[kMaxClasses];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t ncta = lv_ncta(a);
    const uint32_t limit = a.spin_limit;
    for (uint32_t v = blockIdx.x; v < ncta; v += gridDim.x) {
        const uint32_t s = a.cta_seg[v];
        const SegDesc sd = a.seg[s];
        SegState *st = a.st + s;
        const SegArrays ar = seg_arrays(a.sarr, sd);
        LevelClassifier<T> cl;
        __syncthreads();
        load_classifier<T>(cl, a, sd, *st, s_tree, s_spl);
        __syncthreads();
        const uint32_t B = st->B;
        const uint32_t nfs = st->nfull_slots;
        const uint32_t BB = sd.b * T::D;
        unsigned char *base = reinterpret_cast<unsigned char *>(sd.addr);
        const int u = access_unit((uint64_t)(uintptr_t)base);
        const uint32_t W = sd.ncta * (kPermuteThreads / 32);
        const uint32_t wid = (v - sd.cta0) * (kPermuteThreads / 32) + warp;
        uint32_t p = (uint32_t)(((uint64_t)wid * B) / W);
        uint32_t scanned = 0;
        WarpBlock<NV> A, Bk;
#pragma unroll
        for (int c = 0; c < NV; c++) A.v[c] = Bk.v[c] = make_uint4(0, 0, 0, 0);
        uint32_t t = 0;
        bool hold = false;
        bool failed = false;

        while (true) {
            if (!hold) {
                bool got = false;
                while (scanned < B) {
                    // probe the next min(32, B - scanned) buckets with one
                    // read per lane and move to the first that still has
                    // unprocessed blocks (the claim below decides)
                    const uint32_t span = min(32u, B - scanned);
                    bool cand = false;
                    if ((uint32_t)lane < span) {
                        uint32_t q = p + (uint32_t)lane;
                        if (q >= B) q -= B;
                        const unsigned long long vq = *(volatile unsigned long long *)&ar.ptr[q];
                        cand = (int64_t)(uint32_t)vq - (int64_t)kRBias > (int64_t)(vq >> 32);
                    }
                    const uint32_t found = __ballot_sync(0xffffffffu, cand);
                    const uint32_t f = found ? (uint32_t)(__ffs(found) - 1) : span;
                    p += f;
                    if (p >= B) p -= B;
                    scanned += f;
                    if (!found) continue;
                    int res = 0;
                    uint32_t blk = 0;
                    if (lane == 0) {
                        atomicAdd(&ar.readers[p], 1u);
                        __threadfence();
                        unsigned long long old = atomicAdd(&ar.ptr[p], ~0ull);  // r - 1
                        const int64_t w = (int64_t)(old >> 32);
                        const int64_t re = (int64_t)(uint32_t)old - (int64_t)kRBias;
                        if (re > w) {
                            blk = (uint32_t)(re - 1);
                            res = 1;
                        } else {
                            __threadfence();
                            atomicSub(&ar.readers[p], 1u);
                        }
                    }
                    res = __shfl_sync(0xffffffffu, res, 0);
                    if (res) {
                        blk = __shfl_sync(0xffffffffu, blk, 0);
                        if (blk >= nfs) {  // unprocessed blocks are always full slots
                            if (lane == 0) set_status(a.status, IPSGPU_E_INTERNAL);
                            failed = true;
                            break;
                        }
                        warp_load_block<NV>(A, base + (uint64_t)blk * BB, BB, lane, u);
                        __threadfence();
                        __syncwarp();
                        if (lane == 0) atomicSub(&ar.readers[p], 1u);
                        got = true;
                        break;
                    }
                    p = (p + 1 == B) ? 0 : p + 1;
                    scanned++;
                }
                if (!got) break;
                scanned = 0;
                t = cl.warp_class(block_head<T>(A.v[0]), lane);
                hold = true;
            }
            // place the held block into bucket t
            uint32_t slot = 0;
            int unproc = 0;
            if (lane == 0) {
                unsigned long long old = atomicAdd(&ar.ptr[t], 1ull << 32);  // w + 1
                int64_t w = (int64_t)(old >> 32);
                int64_t re = (int64_t)(uint32_t)old - (int64_t)kRBias;
                slot = (uint32_t)w;
                unproc = w < re ? 1 : 0;
            }
            slot = __shfl_sync(0xffffffffu, slot, 0);
            unproc = __shfl_sync(0xffffffffu, unproc, 0);
            if (slot >= ar.dlm[t + 1] || (unproc && slot >= nfs)) {
                // a write pointer never leaves its bucket region
                if (lane == 0) set_status(a.status, IPSGPU_E_INTERNAL);
                failed = true;
                break;
            }
            if (unproc) {
                warp_load_block<NV>(Bk, base + (uint64_t)slot * BB, BB, lane, u);
                const uint32_t t2 = cl.warp_class(block_head<T>(Bk.v[0]), lane);
                if (t2 == t) continue;  // already in place: w moved past it
                warp_store_block<NV>(A, base + (uint64_t)slot * BB, BB, lane, u);
                A = Bk;
                t = t2;
            } else {
                // empty slot: no reader of bucket t may still be copying it out
                int ok = 1;
                if (lane == 0) {
                    __threadfence();
                    ok = bounded_wait_eq(&ar.readers[t], 0u, limit) ? 1 : 0;
                    __threadfence();
                }
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) {
                    if (lane == 0) set_status(a.status, IPSGPU_E_TIMEOUT);
                    failed = true;
                    break;
                }
                if (slot >= nfs) {
                    // the last, partial block of the segment: use the overflow block
                    warp_store_block<NV>(A, seg_ovf(a, sd, T::D), BB, lane, 16);
                    if (lane == 0) st->ovf_used = 1;
                } else {
                    warp_store_block<NV>(A, base + (uint64_t)slot * BB, BB, lane, u);
                }
                hold = false;
            }
        }
        (void)failed;
    }
}

// ---------------------------------------------------------------- cleanup
// For bucket j with element range [lo, hi), region start ds = d_j * b and
// full blocks ending at ws = (d_j + full_j) * b: elements [max(hi, ds),
// min(ws, cap)) of the last full block spill into the next bucket's head;
// they are staged first (k_stage) because the next bucket fills its head
// in k_fill (Sec. 3.1.4, source 1).
template <class T>
__global__ void __launch_bounds__(kAuxThreads) k_stage(LevelArgs a) {
    typedef typename T::E E;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t nseg = lv_nseg(a);
    for (uint32_t s = blockIdx.x; s < nseg; s += gridDim.x) {
        const SegDesc sd = a.seg[s];
        const SegState &st = a.st[s];
        const SegArrays ar = seg_arrays(a.sarr, sd);
        const uint32_t B = st.B, b = sd.b;
        const E *base = reinterpret_cast<const E *>(sd.addr);
        E *stage = reinterpret_cast<E *>(a.arena + sd.stage_off);
        const uint64_t cap = (uint64_t)st.nfull_slots * b;
        for (uint32_t j = warp; j < B; j += blockDim.x / 32) {
            const uint64_t hi = ar.bb[j + 1];
            const uint64_t ds = (uint64_t)ar.dlm[j] * b;
            const uint64_t ws = (uint64_t)(ar.dlm[j] + ar.full[j]) * b;
            const uint64_t lo_o = max(hi, ds), hi_o = min(ws, cap);
            if (hi_o > lo_o && hi_o - lo_o >= b) {  // a spill is shorter than a block
                if (lane == 0) set_status(a.status, IPSGPU_E_INTERNAL);
                continue;
            }
            for (uint64_t x = lo_o + lane; x < hi_o; x += 32)
                stage[(size_t)j * b + (x - lo_o)] = base[x];
        }
    }
}

// One CTA per (segment, class) work item: gather the bucket's missing
// elements from the staged spill, the overflow block and the leftover buffer
// blocks of all stripes, and write them to the bucket's head and tail
// positions (Sec. 3.1.4, sources 1, 2 and 4; the workers of k_permute end
// with empty swap buffers, so source 3 is empty here).  Work item q belongs
// to the segment s with cls0[s] <= q < cls0[s] + C_s.
template <class T>
__global__ void __launch_bounds__(kAuxThreads) k_fill(LevelArgs a) {
    typedef typename T::E E;
    constexpr int kMaxStripePre = 2048;
    __shared__ uint32_t pre[kMaxStripePre + 1];
    __shared__ uint32_t wtmp[34];
    const int tid = threadIdx.x;
    const uint32_t nseg = lv_nseg(a), ncls = lv_ncls(a);
    for (uint32_t q = blockIdx.x; q < ncls; q += gridDim.x) {
        uint32_t lo_s = 0, hi_s = nseg;  // last segment with cls0 <= q
        while (hi_s - lo_s > 1) {
            const uint32_t mid = (lo_s + hi_s) >> 1;
            if (a.seg[mid].cls0 <= q)
                lo_s = mid;
            else
                hi_s = mid;
        }
        const uint32_t s = lo_s;
        const SegDesc sd = a.seg[s];
        const SegState &st = a.st[s];
        const uint32_t j = q - sd.cls0;
        const uint32_t B = st.B, b = sd.b;
        if (j >= B) continue;
        const SegArrays ar = seg_arrays(a.sarr, sd);
        E *base = reinterpret_cast<E *>(sd.addr);
        const uint64_t lo = ar.bb[j], hi = ar.bb[j + 1];
        const uint64_t ds = (uint64_t)ar.dlm[j] * b;
        const uint64_t ws = (uint64_t)(ar.dlm[j] + ar.full[j]) * b;
        const uint64_t cap = (uint64_t)st.nfull_slots * b;
        const uint64_t head_end = min(ds, hi);
        const uint64_t nhead = head_end - lo;
        const uint64_t rend = max(ds, min(min(ws, hi), cap));
        const uint64_t ntail = hi > rend ? hi - rend : 0;
        const uint64_t nfill = nhead + ntail;
        const uint64_t lo_o = max(hi, ds), hi_o = min(ws, cap);
        const uint32_t nstage = hi_o > lo_o ? (uint32_t)min(hi_o - lo_o, (uint64_t)b) : 0;
        // the overflow block holds this bucket's last full block iff the
        // partial slot (index nfull_slots) lies inside [d_j, d_j + full_j)
        const uint32_t novf = (ds <= cap && ws > cap) ? b : 0;
        const E *stage = reinterpret_cast<const E *>(a.arena + sd.stage_off) + (size_t)j * b;
        const E *ovf = reinterpret_cast<const E *>(seg_ovf(a, sd, T::D));
        const uint32_t ns = sd.nstripes;
        uint64_t done = nstage + novf;
        // sources 1 and 4 first
        for (uint64_t t = tid; t < nstage + novf && t < nfill; t += blockDim.x) {
            E x = t < nstage ? stage[t] : ovf[t - nstage];
            uint64_t dst = t < nhead ? lo + t : rend + (t - nhead);
            base[dst] = x;
        }
        // leftover buffer blocks of every stripe, in chunks of kMaxStripePre
        for (uint32_t c0 = 0; c0 < ns; c0 += kMaxStripePre) {
            const uint32_t cn = min((uint32_t)kMaxStripePre, ns - c0);
            for (uint32_t r = tid; r < cn; r += blockDim.x)
                pre[r] = a.scount[a.stripe[sd.stripe0 + c0 + r].cnt_off + j] & (b - 1);
            __syncthreads();
            const uint32_t tot = cta_exclusive_scan<uint32_t>(pre, pre, (int)cn, wtmp);
            if (tid == 0) pre[cn] = tot;
            __syncthreads();
            for (uint32_t t = tid; t < tot; t += blockDim.x) {
                // stripe r with pre[r] <= t < pre[r+1]
                uint32_t l = 0, h = cn;
                while (h - l > 1) {
                    uint32_t mid = (l + h) >> 1;
                    if (pre[mid] <= t)
                        l = mid;
                    else
                        h = mid;
                }
                const StripeDesc &sp = a.stripe[sd.stripe0 + c0 + l];
                const E *left = reinterpret_cast<const E *>(a.arena + sp.left_off) + (size_t)j * b;
                E x = left[t - pre[l]];
                uint64_t tt = done + t;
                if (tt < nfill) {
                    uint64_t dst = tt < nhead ? lo + tt : rend + (tt - nhead);
                    base[dst] = x;
                }
            }
            done += tot;
            __syncthreads();
        }
        if (tid == 0 && done != nfill) set_status(a.status, IPSGPU_E_INTERNAL);
        __syncthreads();
    }
}

// Element-wise classification (the classifier alone, for ipsgpu_classify).
template <class T>
__global__ void __launch_bounds__(kAuxThreads) k_classify_ids(LevelArgs a, uint32_t *out) {
    typedef typename T::K K;
    typedef typename T::E E;
    __shared__ K s_tree[kMaxClasses];
    __shared__ K s_spl[kMaxClasses];
    const SegDesc sd = a.seg[0];
    LevelClassifier<T> cl;
    load_classifier<T>(cl, a, sd, a.st[0], s_tree, s_spl);
    __syncthreads();
    const E *base = reinterpret_cast<const E *>(sd.addr);
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < sd.n;
         i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = cl(base[i]);
}

}  // namespace ipsgpu

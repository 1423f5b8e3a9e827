// Host side of the C ABI declared in include/skmmse.h: argument validation, the
// per-context scratch arena, TMA descriptors, queue construction and the launch of the
// persistent concealment kernel.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "skmmse.h"
#include "skmmse_kernel.cuh"
#include "probe.cuh"

using sk::FrameDev;
using sk::KParams;
using sk::WorkDev;

static_assert(sizeof(sk::TraceRec) == sizeof(skmmse_trace_rec), "trace layout");
// the counter slots map onto the leading long long fields of skmmse_stats, in order
static_assert(offsetof(skmmse_stats, n_beta) == sizeof(long long) * sk::ST_COUNT, "stats layout");
static_assert(SKMMSE_FLAG_IDL_TC == sk::kFlagIdlTc, "flag value");

struct skmmse_context {
    int device = 0;
    int sm_count = 0;
    int blocks_per_sm = 0;
    size_t smem_bytes = 0;
    // device arena
    unsigned char* d_arena = nullptr;
    size_t arena_bytes = 0;
    // fixed device buffers
    int* d_counters = nullptr;               // [0] entries, [1] head, [2] error, [3] pad
    unsigned long long* d_stats = nullptr;   // kNStats
    float* d_ubuf = nullptr;                 // kUbufFloats per persistent CTA (largest grid)
    // pinned staging for frame descriptors and tensor maps
    unsigned char* h_stage = nullptr;
    size_t h_stage_bytes = 0;
    cudaEvent_t stage_done = nullptr;
    bool stage_pending = false;
    long long last_nbeta = 0;
    skmmse_config dflt{0, 64, 64};  // configuration of shape classes not tuned
    std::vector<std::pair<unsigned long long, skmmse_config>> tuned;  // per shape class
    const skmmse_config* forced = nullptr;  // (the autotuner's option under test)
    PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
};

namespace {

constexpr size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

skmmse_status cuda_fail(cudaError_t e) {
    (void)cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? SKMMSE_ERR_NOMEM : SKMMSE_ERR_CUDA;
}

#define SK_CHECK(call)                               \
    do {                                             \
        cudaError_t e_ = (call);                     \
        if (e_ != cudaSuccess) return cuda_fail(e_); \
    } while (0)

skmmse_status validate_params(const skmmse_params* p) {
    if (!p) return SKMMSE_ERR_ARG;
    if (!(p->t_nu > 0.0f) || !(p->sigma2 > 0.0f) || !(p->ridge_rel >= 0.0f) ||
        !(p->beta_tie_rel >= 0.0f) || !std::isfinite(p->t_phi) || !std::isfinite(p->t_nu))
        return SKMMSE_ERR_ARG;
    if (p->ring_step < 1 || p->ring_step > 64) return SKMMSE_ERR_ARG;
    const int nb = p->beta_kmax - p->beta_kmin + 1;
    if (nb < 1 || nb > sk::kMaxBeta || p->beta_kmin < -60 || p->beta_kmax > 60) return SKMMSE_ERR_ARG;
    if (p->precision != SKMMSE_FP32 && p->precision != SKMMSE_MIXED_BF16 &&
        p->precision != SKMMSE_MIXED_FP16)
        return SKMMSE_ERR_ARG;
    if (p->flags & ~(SKMMSE_FLAG_TRACE | SKMMSE_FLAG_FORCE | SKMMSE_FLAG_QUANTIZE | SKMMSE_FLAG_SHORT_WAITS |
                     SKMMSE_FLAG_IDL_TC))
        return SKMMSE_ERR_ARG;
    if ((p->flags & SKMMSE_FLAG_FORCE) && !(p->flags & SKMMSE_FLAG_TRACE)) return SKMMSE_ERR_ARG;
    return SKMMSE_OK;
}

skmmse_status validate_frame(const skmmse_frame& f) {
    if (!f.frame || !f.out) return SKMMSE_ERR_ARG;
    if ((f.mb_lost != nullptr) == (f.px_lost != nullptr)) return SKMMSE_ERR_ARG;  // one mask
    if (f.px_lost && f.px_pitch < f.width) return SKMMSE_ERR_SHAPE;
    if (f.width <= 0 || f.height <= 0 || (f.width & 1) || (f.height & 1)) return SKMMSE_ERR_SHAPE;
    if (f.width > 65536 || f.height > 65536) return SKMMSE_ERR_SHAPE;
    if (f.pitch < f.width || f.out_pitch < f.width) return SKMMSE_ERR_SHAPE;
    if (f.out_f32 && f.out_f32_pitch < f.width) return SKMMSE_ERR_SHAPE;
    if (f.out_f32 && (reinterpret_cast<uintptr_t>(f.out_f32) & 3)) return SKMMSE_ERR_ALIGN;
    if (f.trace && (reinterpret_cast<uintptr_t>(f.trace) & 7)) return SKMMSE_ERR_ALIGN;
    return SKMMSE_OK;
}

KParams make_kparams(const skmmse_params* p) {
    KParams k;
    std::memset(&k, 0, sizeof(k));
    k.t_phi = p->t_phi;
    k.log_t_nu = std::log(p->t_nu);
    k.inv_2sig2 = (float)(1.0 / (2.0 * (double)p->sigma2));
    k.ring_step = p->ring_step;
    // the largest Chebyshev distance between a patch of the block and a candidate patch
    // inside the 48x48 region is 28
    k.nrings = (28 + p->ring_step - 1) / p->ring_step;
    k.ridge_rel = p->ridge_rel;
    k.beta_tie_rel = p->beta_tie_rel;
    k.nbeta = p->beta_kmax - p->beta_kmin + 1;
    for (int b = 0; b < k.nbeta; ++b) {
        const double beta = std::pow(2.0, 0.5 * (p->beta_kmin + b));
        k.inv2beta[b] = (float)(1.0 / (2.0 * beta));
    }
    k.concealed_is_support = p->concealed_is_support ? 1 : 0;
    k.flags = p->flags;
    k.mixed = p->precision;
    k.claim_idle_limit = (p->flags & SKMMSE_FLAG_SHORT_WAITS) ? 64u : (1u << 25);
    k.tile_h13 = 64;
    k.tile_h2 = 64;
    return k;
}


bool config_valid(const skmmse_config& c, int blocks_per_sm) {
    return c.ctas_per_sm >= 0 && c.ctas_per_sm <= blocks_per_sm && (c.tile_cov == 32 || c.tile_cov == 64) &&
           (c.tile_dist == 64 || c.tile_dist == 128);
}

// shape class of a call: precision, profile thresholds, support rule, and the number,
// sizes and mask kinds of its frames (FNV-1a over those values)
unsigned long long shape_key(const skmmse_frame* frames, int n, const skmmse_params* p) {
    unsigned long long h = 1469598103934665603ull;
    auto mix = [&](unsigned long long v) {
        for (int i = 0; i < 8; ++i) {
            h ^= (v >> (8 * i)) & 0xffu;
            h *= 1099511628211ull;
        }
    };
    unsigned tp, tn;
    std::memcpy(&tp, &p->t_phi, 4);
    std::memcpy(&tn, &p->t_nu, 4);
    mix((unsigned long long)p->precision);
    mix(((unsigned long long)tp << 32) | tn);
    mix((unsigned long long)p->concealed_is_support);
    mix((unsigned long long)n);
    for (int i = 0; i < n; ++i)
        mix(((unsigned long long)frames[i].width << 32) | ((unsigned long long)frames[i].height << 1) |
            (frames[i].px_lost ? 1ull : 0ull));
    return h;
}

skmmse_config resolve_config(const skmmse_context* c, const skmmse_frame* frames, int n, const skmmse_params* p) {
    if (c->forced) return *c->forced;
    const unsigned long long k = shape_key(frames, n, p);
    for (const auto& e : c->tuned)
        if (e.first == k) return e.second;
    return c->dflt;
}

// ------------------------------------------------------------------------------------
// kernel instantiations: FP32, and tensor-core contractions with BF16 or FP16 operands

void launch_conceal(const KParams& kp, const WorkDev& w, unsigned grid, cudaStream_t stream) {
    const bool tc = (kp.flags & SKMMSE_FLAG_IDL_TC) != 0u;  // (mixed precision only)
    if (kp.mixed == 1 && tc)
        sk::conceal_kernel<1, true><<<grid, sk::kThreads, sizeof(sk::Smem), stream>>>(w, kp);
    else if (kp.mixed == 2 && tc)
        sk::conceal_kernel<2, true><<<grid, sk::kThreads, sizeof(sk::Smem), stream>>>(w, kp);
    else if (kp.mixed == 1)
        sk::conceal_kernel<1><<<grid, sk::kThreads, sizeof(sk::Smem), stream>>>(w, kp);
    else if (kp.mixed == 2)
        sk::conceal_kernel<2><<<grid, sk::kThreads, sizeof(sk::Smem), stream>>>(w, kp);
    else
        sk::conceal_kernel<0><<<grid, sk::kThreads, sizeof(sk::Smem), stream>>>(w, kp);
}

cudaError_t set_kernel_attributes() {
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(sk::conceal_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(sk::Smem));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(sk::conceal_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(sk::Smem));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(sk::conceal_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(sk::Smem));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(sk::conceal_kernel<1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(sk::Smem));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(sk::conceal_kernel<2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(sk::Smem));
    return e;
}

// ------------------------------------------------------------------------------------
// batch planning shared by direct calls and graph capture

struct BatchLayout {
    long long total_mbs = 0, max_mbs = 1;
    size_t o_frames = 0, o_tmaps = 0, o_eom = 0, o_ent = 0, o_done = 0, o_vals = 0, o_hgt = 0,
           o_bk = 0, o_rem = 0, o_slots = 0, o_mbmask = 0, need = 0, stage_bytes = 0;
    bool any_px = false;
};

skmmse_status plan_batch(const skmmse_frame* frames, int n, const skmmse_params* p, BatchLayout* L) {
    if (n > 65536) return SKMMSE_ERR_SHAPE;
    skmmse_status s = validate_params(p);
    if (s != SKMMSE_OK) return s;
    for (int i = 0; i < n; ++i) {
        s = validate_frame(frames[i]);
        if (s != SKMMSE_OK) return s;
        const long long mbw = (frames[i].width + 15) / 16, mbh = (frames[i].height + 15) / 16;
        L->total_mbs += mbw * mbh;
        if (mbw * mbh > L->max_mbs) L->max_mbs = mbw * mbh;
        if (frames[i].px_lost) L->any_px = true;
    }
    if (L->total_mbs > (1ll << 28)) return SKMMSE_ERR_SHAPE;
    size_t off = 0;
    L->o_frames = off; off = align_up(off + sizeof(FrameDev) * n, 128);
    L->o_tmaps = off; off = align_up(off + sizeof(CUtensorMap) * n, 128);
    L->stage_bytes = off;  // frames + tensor maps come from the host
    L->o_eom = off; off = align_up(off + sizeof(int) * L->total_mbs, 128);
    L->o_ent = off; off = align_up(off + sizeof(int4) * L->total_mbs, 128);
    L->o_done = off; off = align_up(off + sizeof(unsigned) * L->total_mbs, 128);
    L->o_vals = off; off = align_up(off + sizeof(float) * 256 * L->total_mbs, 128);
    L->o_hgt = off; off = align_up(off + sizeof(int) * L->total_mbs, 128);
    L->o_bk = off; off = align_up(off + sizeof(int) * 4 * L->max_mbs, 128);  // off, cnt, head, tail
    L->o_rem = off; off = align_up(off + sizeof(int) * L->total_mbs, 128);
    L->o_slots = off; off = align_up(off + sizeof(int) * L->total_mbs, 128);
    L->o_mbmask = off; off = align_up(off + (L->any_px ? L->total_mbs : 0), 128);  // derived block flags
    L->need = off;
    return SKMMSE_OK;
}

// d_arena: the device arena the descriptors will be used with (the block flags derived
// from a per-pixel mask live there)
void fill_descriptors(PFN_cuTensorMapEncodeTiled_v12000 encode, const skmmse_frame* frames, int n,
                      const skmmse_params* p, const BatchLayout& L, unsigned char* host,
                      unsigned char* d_arena) {
    FrameDev* hf = reinterpret_cast<FrameDev*>(host + L.o_frames);
    CUtensorMap* ht = reinterpret_cast<CUtensorMap*>(host + L.o_tmaps);
    long long mb_base = 0;
    for (int i = 0; i < n; ++i) {
        const skmmse_frame& f = frames[i];
        FrameDev& d = hf[i];
        std::memset(&d, 0, sizeof(d));
        d.in = f.frame;
        d.out = f.out;
        d.out_f32 = f.out_f32;
        d.lost = f.px_lost ? d_arena + L.o_mbmask + mb_base : f.mb_lost;
        d.px_lost = f.px_lost;
        d.px_pitch = f.px_lost ? f.px_pitch : 0;
        d.trace = (p->flags & SKMMSE_FLAG_TRACE) ? f.trace : nullptr;
        d.w = f.width;
        d.h = f.height;
        d.pitch = f.pitch;
        d.out_pitch = f.out_pitch;
        d.out_f32_pitch = f.out_f32 ? f.out_f32_pitch : 0;
        d.mbw = (f.width + 15) / 16;
        d.mbh = (f.height + 15) / 16;
        d.mb_base = (int)mb_base;
        mb_base += (long long)d.mbw * d.mbh;
        std::memset(&ht[i], 0, sizeof(CUtensorMap));
        d.use_tma = 0;
        const bool aligned = (reinterpret_cast<uintptr_t>(f.frame) % 16 == 0) && (f.pitch % 16 == 0);
        if (encode && aligned) {
            cuuint64_t gdim[2] = {(cuuint64_t)f.width, (cuuint64_t)f.height};
            cuuint64_t gstride[1] = {(cuuint64_t)f.pitch};
            cuuint32_t box[2] = {(cuuint32_t)sk::kReg, (cuuint32_t)sk::kReg};
            cuuint32_t estr[2] = {1, 1};
            CUresult r = encode(&ht[i], CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint8_t*>(f.frame),
                                gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            d.use_tma = (r == CUDA_SUCCESS) ? 1 : 0;
        }
    }
}

// the device work of one batch call, in stream order (capturable): received pixels to the
// outputs, counters cleared, queue built, persistent concealment kernel
skmmse_status enqueue_batch(const skmmse_frame* frames, int n, const BatchLayout& L,
                            unsigned char* arena, int* counters, unsigned long long* stats,
                            float* ubuf, const KParams& kp, long long grid, cudaStream_t stream) {
    for (int i = 0; i < n; ++i) {
        const skmmse_frame& f = frames[i];
        if (f.out != f.frame)
            SK_CHECK(cudaMemcpy2DAsync(f.out, f.out_pitch, f.frame, f.pitch, f.width, f.height,
                                       cudaMemcpyDeviceToDevice, stream));
    }
    SK_CHECK(cudaMemsetAsync(counters, 0, 4 * sizeof(int), stream));
    SK_CHECK(cudaMemsetAsync(stats, 0, sk::kNStats * sizeof(unsigned long long), stream));
    SK_CHECK(cudaMemsetAsync(arena + L.o_bk, 0, sizeof(int) * 4 * L.max_mbs, stream));
    SK_CHECK(cudaMemsetAsync(arena + L.o_slots, 0xFF, sizeof(int) * L.total_mbs, stream));
    WorkDev w;
    w.frames = reinterpret_cast<const FrameDev*>(arena + L.o_frames);
    w.tmaps = reinterpret_cast<const CUtensorMap*>(arena + L.o_tmaps);
    w.nframes = n;
    w.entry_of_mb = reinterpret_cast<int*>(arena + L.o_eom);
    w.entries = reinterpret_cast<int4*>(arena + L.o_ent);
    w.counters = counters;
    w.done = reinterpret_cast<unsigned*>(arena + L.o_done);
    w.vals = reinterpret_cast<float*>(arena + L.o_vals);
    w.stats = stats;
    w.height_of_mb = reinterpret_cast<int*>(arena + L.o_hgt);
    w.bk_off = reinterpret_cast<int*>(arena + L.o_bk);
    w.bk_cnt = w.bk_off + L.max_mbs;
    w.bk_head = w.bk_cnt + L.max_mbs;
    w.bk_tail = w.bk_head + L.max_mbs;
    w.rem = reinterpret_cast<int*>(arena + L.o_rem);
    w.slots = reinterpret_cast<int*>(arena + L.o_slots);
    w.nbk = (int)L.max_mbs;
    w.ubuf = ubuf;
    if (L.any_px) {  // block flags of the per-pixel masks, before the queue reads them
        sk::px_block_flags_kernel<<<n, sk::kThreads, 0, stream>>>(w, arena + L.o_mbmask);
        SK_CHECK(cudaGetLastError());
    }
    sk::queue_heights_kernel<<<n, sk::kThreads, 0, stream>>>(w, kp.concealed_is_support);
    sk::queue_offsets_kernel<<<1, sk::kThreads, 0, stream>>>(w);
    sk::queue_fill_kernel<<<n, sk::kThreads, 0, stream>>>(w, kp.concealed_is_support);
    SK_CHECK(cudaGetLastError());
    if (grid > L.total_mbs) grid = L.total_mbs;
    if (grid < 1) grid = 1;
    launch_conceal(kp, w, (unsigned)grid, stream);
    SK_CHECK(cudaGetLastError());
    return SKMMSE_OK;
}

skmmse_status read_stats_from(const unsigned long long* d_stats, const int* d_counters,
                              long long nbeta, skmmse_stats* h, cudaStream_t stream) {
    unsigned long long raw[sk::kNStats];
    int counters[4];
    SK_CHECK(cudaMemcpyAsync(raw, d_stats, sizeof(raw), cudaMemcpyDeviceToHost, stream));
    SK_CHECK(cudaMemcpyAsync(counters, d_counters, sizeof(counters), cudaMemcpyDeviceToHost, stream));
    SK_CHECK(cudaStreamSynchronize(stream));
    std::memset(h, 0, sizeof(*h));
    long long* dst = &h->n_lost_mbs;
    for (int i = 0; i < sk::ST_COUNT; ++i) dst[i] = (long long)raw[i];
    h->n_beta = nbeta;
    h->error = counters[2];
    return counters[2] ? SKMMSE_ERR_TIMEOUT : SKMMSE_OK;
}

// ------------------------------------------------------------------------------------
// Scratch for skmmse_conceal_noalloc(): one file-scope device array, sized for frames of up
// to SKMMSE_NOALLOC_MAX_MBS blocks and a persistent grid of at most SKMMSE_NOALLOC_MAX_CTAS
// CTAs.  Every GPU that loads the library holds it until the process exits.  Layout (byte
// offsets, each 256-aligned): frame descriptor, tensor map, counters + stats, entry_of_mb,
// entries, done flags, per-block values, heights, buckets, dependency counts, ready slots,
// the per-CTA whitened vectors of an HQL step.
constexpr size_t kNaMax = SKMMSE_NOALLOC_MAX_MBS;
constexpr size_t kNaCtas = SKMMSE_NOALLOC_MAX_CTAS;
constexpr size_t kNaFrame = 0;
constexpr size_t kNaTmap = 256;
constexpr size_t kNaCounters = 512;
constexpr size_t kNaStats = 768;
constexpr size_t kNaEom = align_up(kNaStats + sizeof(unsigned long long) * sk::kNStats, 256);
constexpr size_t kNaEnt = align_up(kNaEom + sizeof(int) * kNaMax, 256);
constexpr size_t kNaDone = align_up(kNaEnt + sizeof(int4) * kNaMax, 256);
constexpr size_t kNaVals = align_up(kNaDone + sizeof(unsigned) * kNaMax, 256);
constexpr size_t kNaHgt = align_up(kNaVals + sizeof(float) * 256 * kNaMax, 256);
constexpr size_t kNaBk = align_up(kNaHgt + sizeof(int) * kNaMax, 256);  // off, cnt, head, tail
constexpr size_t kNaRem = align_up(kNaBk + sizeof(int) * 4 * kNaMax, 256);
constexpr size_t kNaSlots = align_up(kNaRem + sizeof(int) * kNaMax, 256);
constexpr size_t kNaUbuf = align_up(kNaSlots + sizeof(int) * kNaMax, 256);
constexpr size_t kNaBytes = align_up(kNaUbuf + sizeof(float) * sk::kUbufFloats * kNaCtas, 256);
static_assert(kNaBytes == SKMMSE_NOALLOC_SCRATCH_BYTES, "static scratch size stated in skmmse.h");
static_assert(sizeof(FrameDev) <= 256 && sizeof(CUtensorMap) <= 256, "scratch header");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

// Writes the frame descriptor and tensor map (passed by value) into the scratch and clears
// what must start at zero: the queue counters and the statistics.
__global__ void noalloc_setup_kernel(FrameDev fd, CUtensorMap tm, unsigned char* scratch) {
    if (threadIdx.x == 0) {
        *reinterpret_cast<FrameDev*>(scratch + kNaFrame) = fd;
        *reinterpret_cast<CUtensorMap*>(scratch + kNaTmap) = tm;
    }
    int* counters = reinterpret_cast<int*>(scratch + kNaCounters);
    unsigned long long* stats = reinterpret_cast<unsigned long long*>(scratch + kNaStats);
    int* bk = reinterpret_cast<int*>(scratch + kNaBk);
    int* slots = reinterpret_cast<int*>(scratch + kNaSlots);
    if (threadIdx.x < 4) counters[threadIdx.x] = 0;
    for (int i = threadIdx.x; i < sk::kNStats; i += blockDim.x) stats[i] = 0ull;
    for (int i = threadIdx.x; i < 4 * (int)kNaMax; i += blockDim.x) bk[i] = 0;
    for (int i = threadIdx.x; i < (int)kNaMax; i += blockDim.x) slots[i] = -1;
}

struct NoAllocDevice {
    bool ready = false;
    unsigned long long ctx_id = 0;     // the primary context the set-up was made in
    unsigned char* scratch = nullptr;  // device address of g_noalloc_scratch on this device
    int sm_count = 0;
    int blocks_per_sm = 0;
    PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
};
constexpr int kNaMaxDevices = 64;
NoAllocDevice g_na_dev[kNaMaxDevices];
std::mutex g_na_mu;

// Unique id of the current context (0 if none is current or the driver cannot tell).  A
// device reset replaces the primary context and with it the scratch address and the kernel
// attributes, so the set-up below is keyed on this id.
unsigned long long current_context_id() {
    using CtxCurrent = CUresult (*)(CUcontext*);
    using CtxId = CUresult (*)(CUcontext, unsigned long long*);
    static CtxCurrent get_current = nullptr;
    static CtxId get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 4000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxCurrent>(fn);
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxId>(fn);
        (void)cudaGetLastError();
        looked_up = true;
    }
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr) return 0;
    if (get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Per device, with that device current, once per primary context: the device address of the
// scratch array (the host-side symbol is only a stand-in), kernel attributes and occupancy.
skmmse_status noalloc_setup(int dev, NoAllocDevice** out) {
    if (dev < 0 || dev >= kNaMaxDevices) return SKMMSE_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_na_mu);
    NoAllocDevice& d = g_na_dev[dev];
    const unsigned long long id = current_context_id();
    if (!d.ready || id == 0 || id != d.ctx_id) {
        d.ready = false;
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);  // makes the primary context current
        if (e != cudaSuccess || ptr == nullptr) return cuda_fail(e);
        e = cudaDeviceGetAttribute(&d.sm_count, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = set_kernel_attributes();
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d.blocks_per_sm, sk::conceal_kernel<0>,
                                                              sk::kThreads, sizeof(sk::Smem));
        if (e != cudaSuccess || d.blocks_per_sm < 1) return cuda_fail(e);
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            d.encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
        (void)cudaGetLastError();
        d.scratch = static_cast<unsigned char*>(ptr);
        d.ctx_id = current_context_id();
        d.ready = true;
    }
    *out = &d;
    return SKMMSE_OK;
}

}  // namespace

extern "C" {

int skmmse_abi_version(void) { return SKMMSE_ABI_VERSION; }

int skmmse_struct_size(int which) {
    switch (which) {
        case 0: return (int)sizeof(skmmse_trace_rec);
        case 1: return (int)sizeof(skmmse_stats);
        case 2: return (int)sizeof(skmmse_params);
        case 3: return (int)sizeof(skmmse_frame);
        case 4: return (int)sizeof(skmmse_config);
        default: return -1;
    }
}

const char* skmmse_status_str(skmmse_status s) {
    switch (s) {
        case SKMMSE_OK: return "ok";
        case SKMMSE_ERR_ARG: return "invalid argument";
        case SKMMSE_ERR_SHAPE: return "unsupported frame shape";
        case SKMMSE_ERR_ALIGN: return "unsupported alignment";
        case SKMMSE_ERR_NOMEM: return "device memory allocation failed";
        case SKMMSE_ERR_CUDA: return "CUDA runtime error";
        case SKMMSE_ERR_TIMEOUT: return "dependency wait timed out on the device";
        case SKMMSE_ERR_UNSUPPORTED: return "unsupported precision or flag";
        case SKMMSE_ERR_TOO_LARGE:
            return "frame exceeds the static scratch of skmmse_conceal_noalloc (SKMMSE_NOALLOC_MAX_MBS blocks)";
        default: return "unknown status";
    }
}

void skmmse_params_preset(skmmse_params* p, int profile) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->t_phi = 20.0f;  // Table I: T_phi = 20 for all profiles
    p->t_nu = profile == SKMMSE_EXPRESS ? 0.01f : profile == SKMMSE_EXCELLENT ? 100.0f : 0.1f;
    p->sigma2 = 10.0f;  // Sec. IV-B
    p->ring_step = 4;
    p->ridge_rel = 1e-3f;
    p->beta_kmin = -8;
    p->beta_kmax = 16;
    p->beta_tie_rel = 1e-3f;
    p->concealed_is_support = 1;
    p->precision = SKMMSE_FP32;
    p->flags = 0;
}

skmmse_status skmmse_create(skmmse_context** out) {
    if (!out) return SKMMSE_ERR_ARG;
    *out = nullptr;
    skmmse_context* c = new (std::nothrow) skmmse_context();
    if (!c) return SKMMSE_ERR_NOMEM;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device);
    c->smem_bytes = sizeof(sk::Smem);
    if (e == cudaSuccess) e = set_kernel_attributes();
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c->blocks_per_sm, sk::conceal_kernel<0>,
                                                          sk::kThreads, c->smem_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_counters, 4 * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_stats, sk::kNStats * sizeof(unsigned long long));
    if (e == cudaSuccess)
        e = cudaMalloc(&c->d_ubuf, sizeof(float) * sk::kUbufFloats * (size_t)c->sm_count * c->blocks_per_sm);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->stage_done, cudaEventDisableTiming);
    if (e == cudaSuccess) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e == cudaSuccess && q == cudaDriverEntryPointSuccess)
            c->encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
        e = cudaSuccess;  // without the entry point every frame takes the plain-load path
    }
    if (e != cudaSuccess || c->blocks_per_sm < 1) {
        skmmse_destroy(c);
        (void)cudaGetLastError();
        return SKMMSE_ERR_CUDA;
    }
    *out = c;
    return SKMMSE_OK;
}

void skmmse_destroy(skmmse_context* c) {
    if (!c) return;
    if (c->stage_pending && c->stage_done) cudaEventSynchronize(c->stage_done);
    if (c->d_arena) cudaFree(c->d_arena);
    if (c->d_counters) cudaFree(c->d_counters);
    if (c->d_stats) cudaFree(c->d_stats);
    if (c->d_ubuf) cudaFree(c->d_ubuf);
    if (c->h_stage) cudaFreeHost(c->h_stage);
    if (c->stage_done) cudaEventDestroy(c->stage_done);
    delete c;
}

skmmse_status skmmse_conceal_batch(skmmse_context* c, const skmmse_frame* frames, int n,
                                   const skmmse_params* p, skmmse_stats* h_stats,
                                   void* stream_v) {
    if (!c || !frames || n < 1) return n < 1 && c && frames ? SKMMSE_ERR_SHAPE : SKMMSE_ERR_ARG;
    BatchLayout L;
    skmmse_status s = plan_batch(frames, n, p, &L);
    if (s != SKMMSE_OK) return s;
    cudaStream_t stream = static_cast<cudaStream_t>(stream_v);
    if (L.need > c->arena_bytes) {
        if (c->stage_pending) cudaEventSynchronize(c->stage_done);
        SK_CHECK(cudaStreamSynchronize(stream));
        if (c->d_arena) cudaFree(c->d_arena);
        c->d_arena = nullptr;
        c->arena_bytes = 0;
        SK_CHECK(cudaMalloc(&c->d_arena, L.need));
        c->arena_bytes = L.need;
    }
    if (L.stage_bytes > c->h_stage_bytes) {
        if (c->stage_pending) cudaEventSynchronize(c->stage_done);
        if (c->h_stage) cudaFreeHost(c->h_stage);
        c->h_stage = nullptr;
        c->h_stage_bytes = 0;
        SK_CHECK(cudaMallocHost(&c->h_stage, L.stage_bytes));
        c->h_stage_bytes = L.stage_bytes;
    }
    if (c->stage_pending) {  // the previous call's upload must have left the staging area
        SK_CHECK(cudaEventSynchronize(c->stage_done));
        c->stage_pending = false;
    }
    fill_descriptors(c->encode, frames, n, p, L, c->h_stage, c->d_arena);
    SK_CHECK(cudaMemcpyAsync(c->d_arena, c->h_stage, L.stage_bytes, cudaMemcpyHostToDevice, stream));
    SK_CHECK(cudaEventRecord(c->stage_done, stream));
    c->stage_pending = true;
    KParams kp = make_kparams(p);
    const skmmse_config cfg = resolve_config(c, frames, n, p);
    kp.tile_h13 = cfg.tile_cov;
    kp.tile_h2 = cfg.tile_dist;
    c->last_nbeta = kp.nbeta;
    const long long grid = (long long)c->sm_count * (cfg.ctas_per_sm > 0 ? cfg.ctas_per_sm : c->blocks_per_sm);
    s = enqueue_batch(frames, n, L, c->d_arena, c->d_counters, c->d_stats, c->d_ubuf, kp, grid, stream);
    if (s != SKMMSE_OK) return s;
    if (h_stats) return skmmse_read_stats(c, h_stats, stream_v);
    return SKMMSE_OK;
}

// ------------------------------------------------------------------------------------
// CUDA graph of a batch call on fixed frame buffers

struct skmmse_graph {
    unsigned char* d_arena = nullptr;
    int* d_counters = nullptr;
    unsigned long long* d_stats = nullptr;
    float* d_ubuf = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    long long nbeta = 0;
};

void skmmse_graph_destroy(skmmse_graph* g) {
    if (!g) return;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    if (g->d_arena) cudaFree(g->d_arena);
    if (g->d_counters) cudaFree(g->d_counters);
    if (g->d_stats) cudaFree(g->d_stats);
    if (g->d_ubuf) cudaFree(g->d_ubuf);
    delete g;
}

skmmse_status skmmse_graph_create(skmmse_context* c, const skmmse_frame* frames, int n,
                                  const skmmse_params* p, skmmse_graph** out) {
    if (!c || !frames || !out || n < 1) return SKMMSE_ERR_ARG;
    *out = nullptr;
    BatchLayout L;
    skmmse_status s = plan_batch(frames, n, p, &L);
    if (s != SKMMSE_OK) return s;
    skmmse_graph* g = new (std::nothrow) skmmse_graph();
    if (!g) return SKMMSE_ERR_NOMEM;
    std::vector<unsigned char> host(L.stage_bytes);
    KParams kp = make_kparams(p);
    const skmmse_config cfg = resolve_config(c, frames, n, p);
    kp.tile_h13 = cfg.tile_cov;
    kp.tile_h2 = cfg.tile_dist;
    g->nbeta = kp.nbeta;
    const long long grid = (long long)c->sm_count * (cfg.ctas_per_sm > 0 ? cfg.ctas_per_sm : c->blocks_per_sm);
    cudaStream_t cs = nullptr;
    cudaError_t e = cudaMalloc(&g->d_arena, L.need);
    if (e == cudaSuccess) fill_descriptors(c->encode, frames, n, p, L, host.data(), g->d_arena);
    if (e == cudaSuccess) e = cudaMalloc(&g->d_counters, 4 * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&g->d_stats, sk::kNStats * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&g->d_ubuf, sizeof(float) * sk::kUbufFloats * (size_t)grid);
    if (e == cudaSuccess) e = cudaMemcpy(g->d_arena, host.data(), L.stage_bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        s = enqueue_batch(frames, n, L, g->d_arena, g->d_counters, g->d_stats, g->d_ubuf, kp, grid, cs);
        cudaGraph_t graph = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
        g->graph = graph;
        if (s == SKMMSE_OK && e2 != cudaSuccess) s = cuda_fail(e2);
        if (s == SKMMSE_OK) {
            e = cudaGraphInstantiate(&g->exec, g->graph, 0);
            if (e != cudaSuccess) s = cuda_fail(e);
        }
    } else {
        s = cuda_fail(e);
    }
    if (cs) cudaStreamDestroy(cs);
    if (s != SKMMSE_OK) {
        skmmse_graph_destroy(g);
        return s;
    }
    *out = g;
    return SKMMSE_OK;
}

skmmse_status skmmse_graph_launch(skmmse_graph* g, void* stream) {
    if (!g || !g->exec) return SKMMSE_ERR_ARG;
    SK_CHECK(cudaGraphLaunch(g->exec, static_cast<cudaStream_t>(stream)));
    return SKMMSE_OK;
}

skmmse_status skmmse_graph_read_stats(skmmse_graph* g, skmmse_stats* h, void* stream_v) {
    if (!g || !h) return SKMMSE_ERR_ARG;
    return read_stats_from(g->d_stats, g->d_counters, g->nbeta, h, static_cast<cudaStream_t>(stream_v));
}

// ------------------------------------------------------------------------------------
// autotuner: persistent CTAs per SM and the tensor-core tile sizes, per shape class

skmmse_status skmmse_autotune(skmmse_context* c, const skmmse_frame* frames, int n,
                              const skmmse_params* p, int reps, void* stream_v, skmmse_config* h_options,
                              float* h_ms, int* h_n_options, int* h_best) {
    if (!c || !frames || n < 1 || reps < 1 || !p) return SKMMSE_ERR_ARG;
    std::vector<skmmse_config> opts;
    const bool mixed = p->precision != SKMMSE_FP32;
    for (int k = 1; k <= c->blocks_per_sm; ++k)
        for (int tc_ : {64, 32})
            for (int td : {64, 128}) {
                if (!mixed && (tc_ != 64 || td != 64)) continue;
                if ((int)opts.size() < SKMMSE_TUNE_MAX_OPTIONS) opts.push_back(skmmse_config{k, tc_, td});
            }
    cudaStream_t stream = static_cast<cudaStream_t>(stream_v);
    cudaEvent_t a = nullptr, b = nullptr;
    SK_CHECK(cudaEventCreate(&a));
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return SKMMSE_ERR_CUDA;
    }
    float best = 1e30f;
    int best_i = 0;
    skmmse_status s = SKMMSE_OK;
    for (int i = 0; i < (int)opts.size() && s == SKMMSE_OK; ++i) {
        c->forced = &opts[i];
        s = skmmse_conceal_batch(c, frames, n, p, nullptr, stream_v);  // warm-up
        float tot = 0.0f;
        for (int r = 0; r < reps && s == SKMMSE_OK; ++r) {
            cudaEventRecord(a, stream);
            s = skmmse_conceal_batch(c, frames, n, p, nullptr, stream_v);
            cudaEventRecord(b, stream);
            if (cudaEventSynchronize(b) != cudaSuccess) s = SKMMSE_ERR_CUDA;
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, a, b);
            tot += ms;
        }
        const float avg = tot / reps;
        if (h_options) h_options[i] = opts[i];
        if (h_ms) h_ms[i] = avg;
        if (avg < best) {
            best = avg;
            best_i = i;
        }
    }
    c->forced = nullptr;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (s != SKMMSE_OK) return s;
    const unsigned long long key = shape_key(frames, n, p);
    bool found = false;
    for (auto& e : c->tuned)
        if (e.first == key) {
            e.second = opts[best_i];
            found = true;
        }
    if (!found) {
        if (c->tuned.size() >= 64) c->tuned.erase(c->tuned.begin());
        c->tuned.emplace_back(key, opts[best_i]);
    }
    if (h_n_options) *h_n_options = (int)opts.size();
    if (h_best) *h_best = best_i;
    return SKMMSE_OK;
}

skmmse_status skmmse_set_config(skmmse_context* c, const skmmse_config* cfg) {
    if (!c || !cfg || !config_valid(*cfg, c->blocks_per_sm)) return SKMMSE_ERR_ARG;
    c->dflt = *cfg;
    return SKMMSE_OK;
}

skmmse_status skmmse_get_config(skmmse_context* c, const skmmse_frame* frames, int n, const skmmse_params* p,
                                skmmse_config* out) {
    if (!c || !frames || n < 1 || !p || !out) return SKMMSE_ERR_ARG;
    *out = resolve_config(c, frames, n, p);
    return SKMMSE_OK;
}

skmmse_status skmmse_set_ctas_per_sm(skmmse_context* c, int k) {
    if (!c || k < 0 || k > c->blocks_per_sm) return SKMMSE_ERR_ARG;
    c->dflt.ctas_per_sm = k;
    return SKMMSE_OK;
}

skmmse_status skmmse_conceal(skmmse_context* c, const uint8_t* d_frame, int width, int height,
                             int pitch, const uint8_t* d_mb_lost, const skmmse_params* p,
                             uint8_t* d_out, int out_pitch, float* d_out_f32,
                             skmmse_stats* h_stats, void* stream) {
    skmmse_frame f;
    std::memset(&f, 0, sizeof(f));
    f.frame = d_frame;
    f.width = width;
    f.height = height;
    f.pitch = pitch;
    f.mb_lost = d_mb_lost;
    f.out = d_out;
    f.out_pitch = out_pitch;
    f.out_f32 = d_out_f32;
    f.out_f32_pitch = width;
    return skmmse_conceal_batch(c, &f, 1, p, h_stats, stream);
}

skmmse_status skmmse_conceal_px(skmmse_context* c, const uint8_t* d_frame, int width, int height,
                                int pitch, const uint8_t* d_px_lost, int px_pitch,
                                const skmmse_params* p, uint8_t* d_out, int out_pitch,
                                float* d_out_f32, skmmse_stats* h_stats, void* stream) {
    skmmse_frame f;
    std::memset(&f, 0, sizeof(f));
    f.frame = d_frame;
    f.width = width;
    f.height = height;
    f.pitch = pitch;
    f.px_lost = d_px_lost;
    f.px_pitch = px_pitch;
    f.out = d_out;
    f.out_pitch = out_pitch;
    f.out_f32 = d_out_f32;
    f.out_f32_pitch = width;
    return skmmse_conceal_batch(c, &f, 1, p, h_stats, stream);
}

skmmse_status skmmse_read_stats(skmmse_context* c, skmmse_stats* h, void* stream_v) {
    if (!c || !h) return SKMMSE_ERR_ARG;
    return read_stats_from(c->d_stats, c->d_counters, c->last_nbeta, h, static_cast<cudaStream_t>(stream_v));
}

skmmse_status skmmse_conceal_noalloc(const uint8_t* d_frame, int width, int height, int pitch,
                                     const uint8_t* d_mb_lost, const skmmse_params* p,
                                     uint8_t* d_out, int out_pitch, float* d_out_f32,
                                     skmmse_stats* h_stats, void* stream_v) {
    skmmse_frame f;
    std::memset(&f, 0, sizeof(f));
    f.frame = d_frame;
    f.width = width;
    f.height = height;
    f.pitch = pitch;
    f.mb_lost = d_mb_lost;
    f.out = d_out;
    f.out_pitch = out_pitch;
    f.out_f32 = d_out_f32;
    f.out_f32_pitch = width;
    skmmse_status s = validate_params(p);
    if (s != SKMMSE_OK) return s;
    if (p->flags & ~SKMMSE_FLAG_QUANTIZE) return SKMMSE_ERR_ARG;  // no trace buffer here
    s = validate_frame(f);
    if (s != SKMMSE_OK) return s;
    const long long mbw = (width + 15) / 16, mbh = (height + 15) / 16;
    if (mbw * mbh > (long long)kNaMax) return SKMMSE_ERR_TOO_LARGE;
    int dev = 0;
    SK_CHECK(cudaGetDevice(&dev));
    NoAllocDevice* nd = nullptr;
    s = noalloc_setup(dev, &nd);
    if (s != SKMMSE_OK) return s;
    cudaStream_t stream = static_cast<cudaStream_t>(stream_v);

    FrameDev fd;
    std::memset(&fd, 0, sizeof(fd));
    fd.in = d_frame;
    fd.out = d_out;
    fd.out_f32 = d_out_f32;
    fd.lost = d_mb_lost;
    fd.trace = nullptr;
    fd.w = width;
    fd.h = height;
    fd.pitch = pitch;
    fd.out_pitch = out_pitch;
    fd.out_f32_pitch = d_out_f32 ? width : 0;
    fd.mbw = (int)mbw;
    fd.mbh = (int)mbh;
    fd.mb_base = 0;
    CUtensorMap tm;
    std::memset(&tm, 0, sizeof(tm));
    const bool aligned = (reinterpret_cast<uintptr_t>(d_frame) % 16 == 0) && (pitch % 16 == 0);
    if (nd->encode && aligned) {
        cuuint64_t gdim[2] = {(cuuint64_t)width, (cuuint64_t)height};
        cuuint64_t gstride[1] = {(cuuint64_t)pitch};
        cuuint32_t box[2] = {(cuuint32_t)sk::kReg, (cuuint32_t)sk::kReg};
        cuuint32_t estr[2] = {1, 1};
        fd.use_tma = nd->encode(&tm, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint8_t*>(d_frame),
                                gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    }
    unsigned char* sc = nd->scratch;
    if (d_out != d_frame)
        SK_CHECK(cudaMemcpy2DAsync(d_out, out_pitch, d_frame, pitch, width, height,
                                   cudaMemcpyDeviceToDevice, stream));
    noalloc_setup_kernel<<<1, sk::kThreads, 0, stream>>>(fd, tm, sc);
    SK_CHECK(cudaGetLastError());
    WorkDev w;
    w.frames = reinterpret_cast<const FrameDev*>(sc + kNaFrame);
    w.tmaps = reinterpret_cast<const CUtensorMap*>(sc + kNaTmap);
    w.nframes = 1;
    w.entry_of_mb = reinterpret_cast<int*>(sc + kNaEom);
    w.entries = reinterpret_cast<int4*>(sc + kNaEnt);
    w.counters = reinterpret_cast<int*>(sc + kNaCounters);
    w.done = reinterpret_cast<unsigned*>(sc + kNaDone);
    w.vals = reinterpret_cast<float*>(sc + kNaVals);
    w.stats = reinterpret_cast<unsigned long long*>(sc + kNaStats);
    w.height_of_mb = reinterpret_cast<int*>(sc + kNaHgt);
    w.bk_off = reinterpret_cast<int*>(sc + kNaBk);
    w.bk_cnt = w.bk_off + kNaMax;
    w.bk_head = w.bk_cnt + kNaMax;
    w.bk_tail = w.bk_head + kNaMax;
    w.rem = reinterpret_cast<int*>(sc + kNaRem);
    w.slots = reinterpret_cast<int*>(sc + kNaSlots);
    w.nbk = (int)(mbw * mbh);
    w.ubuf = reinterpret_cast<float*>(sc + kNaUbuf);
    const KParams kp = make_kparams(p);
    sk::queue_heights_kernel<<<1, sk::kThreads, 0, stream>>>(w, kp.concealed_is_support);
    sk::queue_offsets_kernel<<<1, sk::kThreads, 0, stream>>>(w);
    sk::queue_fill_kernel<<<1, sk::kThreads, 0, stream>>>(w, kp.concealed_is_support);
    SK_CHECK(cudaGetLastError());
    long long grid = (long long)nd->sm_count * nd->blocks_per_sm;
    if (grid > (long long)kNaCtas) grid = (long long)kNaCtas;  // CTAs the static scratch serves
    if (grid > mbw * mbh) grid = mbw * mbh;
    if (grid < 1) grid = 1;
    launch_conceal(kp, w, (unsigned)grid, stream);
    SK_CHECK(cudaGetLastError());
    if (h_stats) {
        unsigned long long raw[sk::kNStats];
        int counters[4];
        SK_CHECK(cudaMemcpyAsync(raw, w.stats, sizeof(raw), cudaMemcpyDeviceToHost, stream));
        SK_CHECK(cudaMemcpyAsync(counters, w.counters, sizeof(counters), cudaMemcpyDeviceToHost, stream));
        SK_CHECK(cudaStreamSynchronize(stream));
        std::memset(h_stats, 0, sizeof(*h_stats));
        long long* dst = &h_stats->n_lost_mbs;
        for (int i = 0; i < sk::ST_COUNT; ++i) dst[i] = (long long)raw[i];
        h_stats->n_beta = kp.nbeta;
        h_stats->error = counters[2];
        if (counters[2]) return SKMMSE_ERR_TIMEOUT;
    }
    return SKMMSE_OK;
}

skmmse_status skmmse_read_phase_clocks(skmmse_context* c, long long* h_clocks16, void* stream_v) {
    if (!c || !h_clocks16) return SKMMSE_ERR_ARG;
    unsigned long long raw[sk::kNPhase];
    SK_CHECK(cudaMemcpyAsync(raw, c->d_stats + sk::kPhaseBase, sizeof(raw), cudaMemcpyDeviceToHost,
                             static_cast<cudaStream_t>(stream_v)));
    SK_CHECK(cudaStreamSynchronize(static_cast<cudaStream_t>(stream_v)));
    for (int i = 0; i < sk::kNPhase; ++i) h_clocks16[i] = (long long)raw[i];
    return SKMMSE_OK;
}


skmmse_status skmmse_probe_peaks(double* h_fma_tflops, double* h_ex2_per_s, void* stream_v) {
    if (!h_fma_tflops || !h_ex2_per_s) return SKMMSE_ERR_ARG;
    cudaStream_t stream = static_cast<cudaStream_t>(stream_v);
    int dev = 0, sms = 0;
    SK_CHECK(cudaGetDevice(&dev));
    SK_CHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * 8, threads = 256;  // 8 CTAs of 256 threads per SM: full occupancy
    float* d_out = nullptr;
    SK_CHECK(cudaMalloc(&d_out, sizeof(float) * blocks * threads));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float ms_fma = 0.0f, ms_ex2 = 0.0f;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // the first round warms up
        cudaEventRecord(e0, stream);
        sk::probe_fma_kernel<<<blocks, threads, 0, stream>>>(d_out, 0.999f, 1e-3f);
        cudaEventRecord(e1, stream);
        e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms_fma, e0, e1);
        if (e != cudaSuccess) break;
        cudaEventRecord(e0, stream);
        sk::probe_ex2_kernel<<<blocks, threads, 0, stream>>>(d_out, 0.5f);
        cudaEventRecord(e1, stream);
        e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms_ex2, e0, e1);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(d_out);
    if (e != cudaSuccess || ms_fma <= 0.0f || ms_ex2 <= 0.0f) return cuda_fail(e);
    const double thr = (double)blocks * threads * sk::kProbeIters * sk::kProbeChains;
    *h_fma_tflops = thr * 2.0 / (ms_fma * 1e-3) / 1e12;
    *h_ex2_per_s = thr / (ms_ex2 * 1e-3);
    return SKMMSE_OK;
}

}  // extern "C"

// SK-MMSE concealment kernel for sm_103a (GB300).
//
// One persistent launch drains a work queue holding every lost 16x16 block of every
// frame of a call.  A CTA of 256 threads owns one block at a time:
//   1. stage the 48x48 support region (the block and its 8 neighbours, Sec. II) into
//      shared memory: received pixels arrive by one TMA tile load of the 8-bit frame,
//      pixels of blocks concealed earlier (when they are support) are read from the
//      per-block FP32 results of the producing CTA after an acquire on its done flag;
//   2. run the sequential fill of the block's 2x2 patches (Sec. II / end of Sec. III),
//      one patch per step, every step parallel across candidates:
//        - next patch: most available pixels in its 6x6 window (ties: lowest index);
//        - context y0, flatness phi (Eq. (17)) and BRL (Eq. (16));
//        - IDL (Eq. (15)) over rings of growing Chebyshev radius with a max-subtracted
//          online softmax and the nu test of Eq. (18) after each ring;
//        - HQL (Eq. (13)): exact covariance, double-float Cholesky and inverse factor,
//          whitened distances, beta grid (Eqs. (9)-(10)), I0 by radix select and the
//          closed-form alpha of Eq. (11);
//        - clip, write back into the support;
//   3. publish the block (release) and fetch the next queue entry.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "df.cuh"
#include "tc.cuh"

namespace sk {

constexpr int kMB = 16;
constexpr int kReg = 48;         // support region side
constexpr int kWin = 6;          // context window side
constexpr int kNpos = kReg - kWin + 1;  // 43 window positions per axis
constexpr int kNcand = kNpos * kNpos;   // 1849
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxNy = 32;
constexpr int kCh = 64;          // HQL candidate chunk
constexpr int kZs = 40;          // staged row: x'(4) y'(32) one(1) pad(3)
constexpr int kZrow = 44;        // row stride of the staged rows (a lane per row: no bank conflicts)
constexpr int kMaxBeta = 32;
constexpr int kMaxI0 = 33;
constexpr int kNStats = 64;
constexpr int kPhaseBase = 48;  // stats slots 48..63: phase clocks (SKMMSE_PHASE_CLOCKS builds)
constexpr int kNPhase = 16;
// whitened context differences u_j = L^-1 (y_j - y0) of one HQL step, kept in global
// memory (per persistent CTA) from the distance pass for the leave-one-out pass: row j of
// 32 floats, its float4 number c4 at float offset ubuf_pos(j, c4) (XOR-swizzled, the
// order of the shared staging rows).  Only the ceil(Ny/4) live groups are written: the
// coordinates past Ny are exact zeros (L^-1 is zero there), and readers take them as such.
constexpr int kUbufFloats = kNcand * kMaxNy;
__host__ __device__ __forceinline__ int ubuf_pos(int j, int c4) { return 4 * (c4 ^ (j & 7)); }

// stats slots (match skmmse_stats field order)
enum {
    ST_LOST = 0, ST_PATCH, ST_EMPTY, ST_BRL, ST_IDL, ST_HQL, ST_NOCAND,
    ST_RING0,  // 16 slots
    ST_IDL_EVALS = ST_RING0 + 16, ST_IDL_NY, ST_HQL_M, ST_HQL_MNY, ST_HQL_I0M, ST_FLOPS,
    ST_HQL_MNY2, ST_HQL_NY3, ST_HQL_I0MNY, ST_PATCH_NY, ST_MMA_FLOPS,
    ST_T_FIRST_INV,  // max over CTAs of ~(start time): the first CTA's start, complemented
    ST_T_LAST,       // max over CTAs of the end time (global timer, ns)
    ST_COUNT
};
static_assert(ST_COUNT <= kPhaseBase, "stats slots");

enum { L_EMPTY = 0, L_BRL = 1, L_IDL = 2, L_HQL = 3, L_NOCAND = 4 };

// Phase clocks: thread 0 of each CTA adds the SM clock cycles spent since its previous
// mark to the slot of the phase that just ended (barrier waits included).  Compiled in
// only with -DSKMMSE_PHASE_CLOCKS; the release build keeps the slots at zero.
enum {
    PH_STAGE = 0, PH_CTX, PH_BRL, PH_IDL, PH_H0, PH_H1, PH_CHOL, PH_H2, PH_H3, PH_H4, PH_H5,
    PH_HFIN, PH_WB, PH_PUB, PH_X1, PH_X2  // X1, X2: spare slots for finer splits
};
#ifdef SKMMSE_PHASE_CLOCKS
#define SK_PHASE(slot)                                           \
    do {                                                         \
        if (threadIdx.x == 0) {                                  \
            const long long t_ = clock64();                      \
            sm.st[kPhaseBase + (slot)] += (unsigned long long)(t_ - sm.ph_t); \
            sm.ph_t = t_;                                        \
        }                                                        \
    } while (0)
#else
#define SK_PHASE(slot) \
    do {               \
    } while (0)
#endif

struct KParams {
    float t_phi;
    float log_t_nu;
    float inv_2sig2;      // 1 / (2 sigma^2)
    int ring_step;
    int nrings;
    float ridge_rel;
    float beta_tie_rel;
    int nbeta;
    float inv2beta[kMaxBeta];  // 1 / (2 beta_b), beta_b = 2^((kmin+b)/2)
    int concealed_is_support;
    unsigned flags;
    int mixed;            // 0: FP32 on the CUDA cores; 1: BF16, 2: FP16 tensor-core contractions
    unsigned claim_idle_limit;  // polls without progress before a CTA gives up claiming
    int tile_h13;         // candidates per chunk of the covariance pass: 32 or 64
    int tile_h2;          // candidates per tile of the distance pass: 64 or 128 (MMA M)
};

struct FrameDev {
    const uint8_t* in;
    uint8_t* out;
    float* out_f32;
    const uint8_t* lost;      // block flags (given, or derived from px_lost)
    void* trace;
    const uint8_t* px_lost;   // per-pixel loss (arbitrarily shaped), or null: whole blocks
    int w, h, pitch, out_pitch, out_f32_pitch;
    int mbw, mbh;
    int mb_base;  // offset of this frame's blocks in entry_of_mb
    int use_tma;
    int px_pitch;
    int pad[2];
};

struct WorkDev {
    const FrameDev* frames;
    const CUtensorMap* tmaps;
    int nframes;
    int* entry_of_mb;         // per block of all frames: queue entry or -1
    int4* entries;            // (frame, block index, rank among the frame's lost blocks, bucket)
    int* counters;            // [0] entries, [1] claimed, [2] error word, [3] first live bucket
    unsigned* done;           // per entry: 0 pending, 1 done, 2 done with error
    float* vals;              // per entry: 256 unrounded values of the block
    unsigned long long* stats;
    int* height_of_mb;        // per block of all frames: longest chain of dependants (-1 received,
                              // kIsolated for a lost block with no lost neighbour)
    int* bk_off;              // per bucket: number of entries, then the bucket's first entry
    int* bk_cnt;              // per bucket: entries handed out while filling (= its size after)
    int* bk_head;             // per bucket: ready entries claimed
    int* bk_tail;             // per bucket: ready entries published
    int* rem;                 // per entry: dependencies not yet done
    int* slots;               // per entry position: the ready entries of each bucket, -1 until published
    int nbk;                  // buckets allocated (>= blocks of the largest frame)
    float* ubuf;              // per persistent CTA (blockIdx.x): kUbufFloats, u_j of the HQL step
};

struct TraceRec {             // layout of skmmse_trace_rec
    int32_t mb;
    int16_t step, patch;
    int8_t layer, ring, beta_idx, n0;
    int16_t ny, m;
    float phi, log_nu, alpha, eps_best;
    float x[4];
    uint16_t i0[36];
};

// ------------------------------------------------------------------------------------
// shared memory

struct __align__(16) HqlP1 {                 // covariance / factorisation phase
    int cint[36][36];
    float cfrac[36][36];
    df32 A[32][33];
    df32 X[32][33];
};
constexpr int kI0Pad = 36;   // leave-one-out members padded to whole 3-member tiles
constexpr int kWb = 44;      // leave-one-out candidate buffer row: x'(4) G u(4) pad(4) u(32)
struct __align__(16) HqlP2 {                 // beta phase (CUDA-core form)
    float mrg[kThreads][37];                 // per-thread partial sums before a merge
};

struct __align__(16) Hql {
    uint16_t cand[kNcand + 7];  // window top-left as S offset u*48+v
    float d[kNcand + 7];
    __align__(16) float Linv[32][36];
    float G[4][32];
    df32 cxy[4][32];            // C_XY (double-float)
    df32 K[4][32];              // C_XY C_YY^-1 (double-float)
    __align__(16) float Kf[4][36];  // K rounded to FP32 (rows padded: conflict-free column reads)
    __align__(16) float ys[36];  // y0 - shift (compacted)
    short off[36];              // compacted context offsets rel. window top-left
    int i0[kMaxI0];             // I0 candidate indices, ascending
    float dmin;
    int M, n0, bstar;
    float eps[kMaxBeta];
    df32 ebard[32];
    df32 xt0d[4];
    df32 corr[4];
    float red[kWarps][4];
    int scan[kWarps + 1];
    int hist[2][256];  // I0 radix select: this pass's histogram, the next pass's cleared
    int sel[2][2];
    int colNi[36];
    float colF[36];
    int koff[kZs];
    float lam;
    float alpha;
    __align__(16) float UI[kI0Pad][36];      // whitened I0 members, u_i = L^-1 (y_i - y0)
    float XI[kMaxI0][4];                     // x_i - shift of the I0 members
    float accI[kMaxI0][12];                  // merged leave-one-out sums: x'(4) G u(4) sum w
    union {
        df32 accBd[kMaxBeta][kZs];  // beta-pass sums (double-float), end of H3 only
        struct {  // CUDA-core staging and phase buffers
            __align__(16) float Z[2][kCh][kZrow];  // staged candidates, centred by the integer shift
            union {
                HqlP1 p1;
                HqlP2 p2;
            };
        };
        // tensor-core operand tiles (64 KB; layout in tl::).  128-byte aligned in shared memory:
        // a core matrix (8 rows of 16 bytes) then fills one 128-byte line, which the tensor
        // core reads in one pass (at a 64-byte offset the passes measured ~1.6x slower)
        __align__(128) uint16_t mx[32768];
        struct {  // leave-one-out pass: per-warp candidate buffers and the warps' partial sums
            __align__(16) float Wb[kWarps][32][kWb];
            float Mg[kWarps][33][10];
        } h5;
    };
};

struct __align__(16) IdlSlot {
    float m, s0, sx[4];
    int cnt;
    int pad;
};

struct __align__(128) Smem {
    uint8_t raw[kReg * kReg];          // TMA destination (2304 B)
    unsigned long long mbar;
    unsigned long long av[kReg];       // availability bits per region row
    unsigned long long unfilled;       // patches still to fill
    float S[kReg * kReg];              // support values (0 where unavailable)
    int nbst[9];                       // neighbour status: 0 received, 1 concealed, 2 n/a
    int nbent[9];
    int entry;
    int pad0;
    struct {
        unsigned long long ymask;
        int step, pa, pb, ny;
        float phi, mean;
    } hand;                            // step handed from warp 0 to the CTA
    unsigned long long st[kNStats];    // per-CTA counters
    TraceRec tr;                       // trace record of the current step
    long long ph_t;                    // last phase mark (SKMMSE_PHASE_CLOCKS)
    uint64_t mma_bar;                  // tensor-core completion (mixed precision)
    unsigned tmem_base;                // tensor memory of this CTA (mixed precision)
    int mma_err;
    union {
        IdlSlot idl[2][kWarps];
        Hql hql;
    };
    uint8_t order[64];                 // fill order of the block (patch of each step)
};

// ------------------------------------------------------------------------------------
// small helpers

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int ld_acquire_i(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_relaxed_i(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_i(int* p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// bounded wait on an mbarrier phase; returns false if the bound was reached
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity,
                                          unsigned max_iter) {
    const unsigned a = smem_u32(bar);
    for (unsigned it = 0; it < max_iter; ++it) {
        unsigned ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
        if (it > 64) __nanosleep(128);
    }
    return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map,
                                            unsigned long long* bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tmap_acquire(const CUtensorMap* map) {
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(map) : "memory");
}

// the GPU's global timer (nanoseconds), comparable across the CTAs and launches of a device
__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// block-wide exclusive scan of one int per thread; returns the prefix, *total = sum
__device__ __forceinline__ int block_exscan(int v, int* scratch /*kWarps+1*/, int* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) scratch[wid] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int w = 0; w < kWarps; ++w) {
            int t = scratch[w];
            scratch[w] = run;
            run += t;
        }
        scratch[kWarps] = run;
    }
    __syncthreads();
    const int r = scratch[wid] + x - v;
    *total = scratch[kWarps];
    __syncthreads();
    return r;
}

// context of the current step, held by every thread
struct StepCtx {
    int pa, pb;          // patch row/column inside the block
    int wr, wc;          // window top-left in region coordinates
    unsigned long long ymask;  // 36 bits, window raster order
    unsigned rowcfg[6];  // per window row: context bits | x bits
    int ny;
    float phi, mean;
    float y0w[36];       // window values (0 where unavailable)
};

// candidate window (u, v) valid: every configured position available (the six rows read
// at once, no early exit)
__device__ __forceinline__ bool cand_valid(const Smem& sm, const StepCtx& c, int u, int v) {
    unsigned missing = 0u;
#pragma unroll
    for (int r = 0; r < 6; ++r) missing |= c.rowcfg[r] & ~((unsigned)(sm.av[u + r] >> v) & 63u);
    return missing == 0u;
}

// squared Euclidean context distance of window (base = u*48+v), Eq. (15).  All 36 window
// values are read (the window lies inside the region); a position outside the context adds
// fma(0, 0, d) = d exactly (the partial sums are never -0), so the sums are those of the
// context positions alone, without a branch per position.
__device__ __forceinline__ float ctx_dist(const float* S, const StepCtx& c, int base) {
    float d[4] = {0.0f, 0.0f, 0.0f, 0.0f};  // four partial sums: independent FMA chains
#pragma unroll
    for (int k = 0; k < 36; ++k) {
        const float diff = c.y0w[k] - S[base + (k / 6) * kReg + (k % 6)];
        const float t = ((c.ymask >> k) & 1ull) ? diff : 0.0f;
        d[k & 3] = __fmaf_rn(t, t, d[k & 3]);
    }
    return (d[0] + d[1]) + (d[2] + d[3]);
}

// ring k (1-based) enumeration: i-th position of the square annulus with Chebyshev
// radius in (rin, rout] around the origin
__device__ __forceinline__ void annulus_pos(int i, int rin, int rout, int* dy, int* dx) {
    const int side = 2 * rout + 1, t = rout - rin, top = t * side;
    if (i < top) {
        *dy = -rout + i / side;
        *dx = -rout + i % side;
    } else if (i < 2 * top) {
        const int q = i - top;
        *dy = rin + 1 + q / side;
        *dx = -rout + q % side;
    } else {
        const int q = i - 2 * top;
        const int row = q / (2 * t), cc = q % (2 * t);
        *dy = -rin + row;
        *dx = cc < t ? -rout + cc : rin + 1 + (cc - t);
    }
}

// (the rescale as a select: the factor is exactly 1 unless s is a new maximum; its products
// rounded on their own, as in the branch form)
__device__ __forceinline__ void online_add(float s, float x0, float x1, float x2, float x3,
                                           float& m, float& s0, float sx[4]) {
    const float e = __expf(m - s);
    const float sc = s > m ? e : 1.0f;
    s0 = __fmul_rn(s0, sc);
#pragma unroll
    for (int q = 0; q < 4; ++q) sx[q] = __fmul_rn(sx[q], sc);
    m = fmaxf(m, s);
    const float w = __expf(s - m);
    s0 += w;
    sx[0] = __fmaf_rn(w, x0, sx[0]);
    sx[1] = __fmaf_rn(w, x1, sx[1]);
    sx[2] = __fmaf_rn(w, x2, sx[2]);
    sx[3] = __fmaf_rn(w, x3, sx[3]);
}

constexpr float kNegBig = -1.0e30f;

// ------------------------------------------------------------------------------------
// IDL: Eq. (15) over growing rings; returns 1 accepted, 0 not accepted, -1 no candidate

struct CtxStats {
    unsigned long long ymask;  // context positions, window raster order (the patch excluded)
    int ny;
    float phi, mean;  // flatness (max - min) and mean of the context, Eqs. (16)-(17)
};

// context of the window at (wr, wc): size, flatness and mean.  Warp-level reductions; every
// lane returns the same values.  Lane l takes window position l (raster order) and lanes
// 0..3 also position 32 + l; both positions' availability rows and values are read at once
// (the values unconditionally: they lie inside the region).  Support values lie in
// [0, 255] (clipped estimates, 8-bit pixels), where the order of the FP32 bit patterns
// (with -0 folded to +0) is the order of the values: the maximum and minimum are single
// integer warp reductions.  The sum adds each lane's one or two values, then a butterfly
// over the lanes: a fixed order of FP32 additions.
__device__ __forceinline__ CtxStats ctx_stats(const Smem& sm, int wr, int wc, int lane) {
    const int r0 = lane / 6, c0 = lane - 6 * (lane / 6);  // position lane (rows 0..5)
    const int c1 = 2 + (lane & 3);                        // position 32 + lane: row 5
    const bool own = (r0 == 2 || r0 == 3) && (c0 == 2 || c0 == 3);  // the patch: never context
    const unsigned long long row0 = sm.av[wr + r0], row1 = sm.av[wr + 5];
    const float v0 = sm.S[(wr + r0) * kReg + wc + c0];
    const float v1 = sm.S[(wr + 5) * kReg + wc + c1];
    const bool on0 = !own && ((row0 >> (wc + c0)) & 1ull);
    const bool on1 = lane < 4 && ((row1 >> (wc + c1)) & 1ull);
    const unsigned b0 = __float_as_uint(v0 + 0.0f), b1 = __float_as_uint(v1 + 0.0f);  // -0 -> +0
    unsigned mxb = on0 ? b0 : 0u, mnb = on0 ? b0 : 0xFFFFFFFFu;
    if (on1) {
        mxb = max(mxb, b1);
        mnb = min(mnb, b1);
    }
    float sum = on0 ? 0.0f + v0 : 0.0f;
    if (on1) sum += v1;
    const unsigned bal0 = __ballot_sync(0xffffffffu, on0), bal1 = __ballot_sync(0xffffffffu, on1);
    const int ny = __popc(bal0) + __popc(bal1);
    mxb = __reduce_max_sync(0xffffffffu, mxb);
    mnb = __reduce_min_sync(0xffffffffu, mnb);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    CtxStats cs;
    cs.ymask = (unsigned long long)bal0 | ((unsigned long long)bal1 << 32);
    cs.ny = ny;
    cs.phi = ny > 0 ? __uint_as_float(mxb) - __uint_as_float(mnb) : 0.0f;
    cs.mean = ny > 0 ? sum / (float)ny : 0.0f;
    return cs;
}

// The dynamic shared memory of the concealment kernel.  Out-of-line device functions take
// their view of it from here rather than through a reference argument, so that the
// compiler keeps every access in the shared address space.
extern __shared__ __align__(128) unsigned char smem_raw[];
__device__ __forceinline__ Smem& smem_ref() { return *reinterpret_cast<Smem*>(smem_raw); }

// Fill order of a block (R2: the unfilled patch with the most available pixels in its 6x6
// window less the patch itself, ties to the lowest index).  It depends on availability only,
// so warp 0 simulates it once when the block is staged.  Lane l holds patches l and l + 32
// and their counts.  Filling patch p makes its unavailable pixels available; those lie in
// the windows of exactly the 8 neighbouring patches (the window of q spans patch rows and
// columns q +- 1), whose counts grow by that number.  order[s] = the patch of step s.
__device__ __noinline__ void fill_order(int npatch) {
    Smem& sm = smem_ref();
    const int lane = threadIdx.x & 31;
    const unsigned long long uf0 = sm.unfilled;
    int cnt[2], newpx[2];
    bool uf[2];
#pragma unroll
    for (int h2 = 0; h2 < 2; ++h2) {
        const int p = lane + 32 * h2;
        const int a = p >> 3, b = p & 7;
        const int wr = kMB + 2 * a - 2, wc = kMB + 2 * b - 2;
        int c = 0;
#pragma unroll
        for (int r = 0; r < 6; ++r)
            c += __popc((unsigned)(sm.av[wr + r] >> wc) & ((r == 2 || r == 3) ? 0x33u : 63u));
        cnt[h2] = c;
        newpx[h2] = 4 - __popc((unsigned)(sm.av[wr + 2] >> (wc + 2)) & 3u) -
                    __popc((unsigned)(sm.av[wr + 3] >> (wc + 2)) & 3u);
        uf[h2] = ((uf0 >> p) & 1ull) != 0ull;
    }
    for (int s = 0; s < npatch; ++s) {
        int key = -1;
#pragma unroll
        for (int h2 = 0; h2 < 2; ++h2)
            if (uf[h2]) key = max(key, cnt[h2] * 64 + (63 - (lane + 32 * h2)));
        const int best = __reduce_max_sync(0xffffffffu, key);
        const int ps = 63 - (best & 63);
        const int np = __shfl_sync(0xffffffffu, (ps >> 5) ? newpx[1] : newpx[0], ps & 31);
        if (lane == 0) sm.order[s] = (uint8_t)ps;
        const int as = ps >> 3, bs = ps & 7;
#pragma unroll
        for (int h2 = 0; h2 < 2; ++h2) {
            const int p = lane + 32 * h2;
            const int da = (p >> 3) - as, db = (p & 7) - bs;
            if (p == ps) uf[h2] = false;
            else if (da >= -1 && da <= 1 && db >= -1 && db <= 1) cnt[h2] += np;
        }
    }
    __syncwarp();
}


// Not inlined, with scalar arguments: the 36 context values live in registers only while
// this function runs, so the per-step loop of the kernel keeps a small register footprint.
struct IdlOut {
    float x[4];
    float lognu;
    int ring;
    int evals;  // candidates evaluated (thread 0)
    int r;      // 1 accepted, 0 not accepted, -1 no candidate
};

template <bool BF16>
__device__ __noinline__ void idl_tc_distances(int wr, int wc, unsigned long long ymask, float cen,
                                              uint32_t tmem, uint32_t mph);
constexpr unsigned kFlagIdlTc = 16u;  // SKMMSE_FLAG_IDL_TC

// IDLTC: the kernel instantiation with the tensor-core distances for the rings after the
// first (SKMMSE_FLAG_IDL_TC); the default instantiation carries none of that code
template <int MIXED, bool IDLTC>
__device__ __forceinline__ IdlOut idl_step(const KParams& P, int wr, int wc,
                                        unsigned long long ymask, int ny, float mean, uint32_t mph) {
    Smem& sm = smem_ref();
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    StepCtx c;
    c.wr = wr;
    c.wc = wc;
    c.ymask = ymask;
    c.ny = ny;
    c.mean = mean;
#pragma unroll
    for (int r = 0; r < 6; ++r)
        c.rowcfg[r] = (unsigned)((ymask >> (6 * r)) & 63ull) | ((r == 2 || r == 3) ? 12u : 0u);
#pragma unroll
    for (int k = 0; k < 36; ++k) c.y0w[k] = sm.S[(wr + k / 6) * kReg + wc + k % 6];
    IdlOut out;
    float* xhat = out.x;
    xhat[0] = xhat[1] = xhat[2] = xhat[3] = mean;
    const int pr = c.wr + 2, pc = c.wc + 2;  // patch top-left (region)
    const float inv_h = P.inv_2sig2 / (float)c.ny;
    const float cen = rintf(c.mean);
    float m = kNegBig, s0 = 0.0f, sx[4] = {0.f, 0.f, 0.f, 0.f};
    int cnt = 0;
    int accepted = 0, k = 1;
    float lognu = -INFINITY;
    int total_cnt = 0;
    // IDLTC (mixed precision): the rings after the first take their distances from one
    // tensor-core pass over every window position
    for (k = 1; k <= P.nrings; ++k) {
        const int rin = (k - 1) * P.ring_step, rout = k * P.ring_step;
        const int side = 2 * rout + 1, inner = 2 * rin + 1;
        const int npos = side * side - inner * inner;
        if constexpr (IDLTC && MIXED != 0) {
            if (k == 2) idl_tc_distances<MIXED == 1>(c.wr, c.wc, c.ymask, cen, sm.tmem_base, mph);
        }
        const bool from_d = IDLTC && k >= 2;
        for (int i = tid; i < npos; i += kThreads) {
            int dy, dx;
            annulus_pos(i, rin, rout, &dy, &dx);
            const int u = pr + dy - 2, v = pc + dx - 2;
            if (u < 0 || v < 0 || u >= kNpos || v >= kNpos) continue;
            if (!cand_valid(sm, c, u, v)) continue;
            const int base = u * kReg + v;
            const float d = from_d ? sm.hql.d[u * kNpos + v] : ctx_dist(sm.S, c, base);
            const float* X = &sm.S[base + 2 * kReg + 2];
            online_add(-d * inv_h, X[0] - cen, X[1] - cen, X[kReg] - cen, X[kReg + 1] - cen, m,
                       s0, sx);
            ++cnt;
        }
        // warp combine: the maximum first, then one rescale per lane and plain sums.  The
        // scores are <= 0 (or kNegBig): with the sign bit forced, their bit patterns order
        // inversely to the values, so the maximum is one unsigned minimum reduction.
        const float wm = __uint_as_float(__reduce_min_sync(0xffffffffu, __float_as_uint(m) | 0x80000000u));
        const float lsc = __expf(m - wm);
        float ws = s0 * lsc, wx[4] = {sx[0] * lsc, sx[1] * lsc, sx[2] * lsc, sx[3] * lsc};
        const int wc = __reduce_add_sync(0xffffffffu, cnt);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            ws += __shfl_xor_sync(0xffffffffu, ws, o);
#pragma unroll
            for (int q = 0; q < 4; ++q) wx[q] += __shfl_xor_sync(0xffffffffu, wx[q], o);
        }
        IdlSlot* slot = &sm.idl[k & 1][0];
        if (lane == 0) {
            slot[wid].m = wm;
            slot[wid].s0 = ws;
#pragma unroll
            for (int q = 0; q < 4; ++q) slot[wid].sx[q] = wx[q];
            slot[wid].cnt = wc;
        }
        __syncthreads();
        // CTA combine, the same way over the warps' slots
        float bm = slot[0].m;
#pragma unroll
        for (int w = 1; w < kWarps; ++w) bm = fmaxf(bm, slot[w].m);
        float bs = 0.0f, bx[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        int bc = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            const float e = __expf(slot[w].m - bm);
            bs = __fmaf_rn(slot[w].s0, e, bs);
#pragma unroll
            for (int q = 0; q < 4; ++q) bx[q] = __fmaf_rn(slot[w].sx[q], e, bx[q]);
            bc += slot[w].cnt;
        }
        total_cnt = bc;
        if (bc > 0) {
            lognu = bm + logf(bs);
            if (lognu >= P.log_t_nu) {
                accepted = 1;
                const float inv = 1.0f / bs;
#pragma unroll
                for (int q = 0; q < 4; ++q) xhat[q] = cen + bx[q] * inv;
                break;
            }
        }
    }
    out.evals = total_cnt;
    out.ring = accepted ? k : P.nrings;
    out.lognu = lognu;
    out.r = total_cnt == 0 ? -1 : accepted;
    return out;
}

// ------------------------------------------------------------------------------------
// HQL

// per-column source of a staged candidate row: S offset relative to the window top-left,
// or -1 (zero padding), -2 (the constant-one column)
__device__ __forceinline__ void hql_build_koff(Hql& h, int nz) {
    const int tid = threadIdx.x;
    if (tid < kZs) {
        int o = -1;
        if (tid < nz) o = (tid < 4) ? (tid >> 1) * kReg + (tid & 1) + 2 * kReg + 2 : h.off[tid - 4];
        else if (tid == 36) o = -2;
        h.koff[tid] = o;
    }
}

// stage candidates [c0, c0+n) into Z[buf]: x' (4), y' (ny), 1, zero padding.  Thread t
// fills columns 10 (t & 3) .. +9 of candidate rows t >> 2 (and + 64 when kCh > 64): one
// candidate offset per row and ten independent loads.
__device__ __forceinline__ void hql_stage(Smem& sm, int buf, int c0, int n, float shift) {
    static_assert(kZs == 40 && kThreads == 256 && kCh == 64, "staging layout");
    Hql& h = sm.hql;
    const int j = threadIdx.x >> 2, k0 = 10 * (threadIdx.x & 3);
    const bool live = j < n;
    const int cb = live ? h.cand[c0 + j] : 0;
    float v[10];
#pragma unroll
    for (int t = 0; t < 10; ++t) {
        const int o = h.koff[k0 + t];
        float x = 0.0f;
        if (live) {
            if (o >= 0) x = sm.S[cb + o] - shift;
            else if (o == -2) x = 1.0f;
        }
        v[t] = x;
    }
    float* dst = &h.Z[buf][j][k0];
#pragma unroll
    for (int t = 0; t < 10; t += 2) *reinterpret_cast<float2*>(dst + t) = make_float2(v[t], v[t + 1]);
}

// stage the integer parts (as int) into Z[0] and the fractions into Z[1]; returns whether
// this thread saw a non-integer value
__device__ __forceinline__ bool hql_stage_split(Smem& sm, int c0, int n, float shift) {
    Hql& h = sm.hql;
    bool frac = false;
    int* zi = reinterpret_cast<int*>(&h.Z[0][0][0]);
    float* zf = &h.Z[1][0][0];
#pragma unroll 2
    for (int idx = threadIdx.x; idx < kCh * kZs; idx += kThreads) {
        const int j = idx / kZs, k = idx - j * kZs;
        const int o = h.koff[k];
        float v = 0.0f;
        if (j < n && o >= 0) v = sm.S[h.cand[c0 + j] + o] - shift;
        const float nv = rintf(v);
        zi[j * kZrow + k] = __float2int_rn(nv);
        zf[j * kZrow + k] = v - nv;
        frac = frac || (v != nv);
    }
    return frac;
}

// whitened coordinates of candidates tj, tj+1 (rows of Z[buf]), coordinates 4tq..4tq+3:
// u = L^-1 (y_j - y0)
__device__ __forceinline__ void whiten_tile(const Hql& h, int buf, int ny, int tj, int tq,
                                            float u0[4], float u1[4]) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        u0[q] = 0.0f;
        u1[q] = 0.0f;
    }
    for (int l4 = 0; l4 <= tq; ++l4) {
        if (4 * l4 >= ny) break;
        const float4 e0v = *reinterpret_cast<const float4*>(&h.Z[buf][tj][4 + 4 * l4]);
        const float4 e1v = *reinterpret_cast<const float4*>(&h.Z[buf][tj + 1][4 + 4 * l4]);
        const float4 ysv = *reinterpret_cast<const float4*>(&h.ys[4 * l4]);
        const float e0[4] = {e0v.x - ysv.x, e0v.y - ysv.y, e0v.z - ysv.z, e0v.w - ysv.w};
        const float e1[4] = {e1v.x - ysv.x, e1v.y - ysv.y, e1v.z - ysv.z, e1v.w - ysv.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 lv = *reinterpret_cast<const float4*>(&h.Linv[4 * tq + q][4 * l4]);
            const float L4[4] = {lv.x, lv.y, lv.z, lv.w};
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                u0[q] = __fmaf_rn(L4[r], e0[r], u0[q]);
                u1[q] = __fmaf_rn(L4[r], e1[r], u1[q]);
            }
        }
    }
}

// ------------------------------------------------------------------------------------
// Mixed precision: the HQL contractions on tcgen05 tensor cores.  Operands are split into
// two 16-bit parts, v ~ hi + lo (BF16: ~16 significant bits; FP16: ~22), and every product
// is accumulated as hi*hi + hi*lo + lo*hi in FP32 tensor memory.

// The splits stay off the format-conversion unit, which runs at a fraction of the FP32 rate
// and set the staging time of the passes:
//   BF16: round-to-nearest-even on the FP32 bits with integer operations (exact);
//   FP16: the high part is v rounded to 11 significant bits by Veltkamp's splitting in FP32
//         (non-contracting intrinsics), the low part v - hi exactly, and each pair of values
//         is converted by one packed conversion.
__device__ __forceinline__ uint32_t bf16_bits_rn(float v) {  // finite v
    const uint32_t u = __float_as_uint(v);
    return (u + 0x7FFFu + ((u >> 16) & 1u)) >> 16;
}

__device__ __forceinline__ float veltkamp_hi11(float v) {  // v to 11 significant bits
    const float g = __fmul_rn(8193.0f, v);  // 2^13 + 1
    return __fadd_rn(g, __fsub_rn(v, g));
}

__device__ __forceinline__ uint32_t pack_f16x2(float a, float b) {  // a low, b high, RN
    const __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
}

// the pair (v0, v1) as packed high halves and packed low halves
template <bool BF16>
__device__ __forceinline__ void split2(float v0, float v1, uint32_t& hi2, uint32_t& lo2) {
    if (BF16) {
        const uint32_t h0 = bf16_bits_rn(v0), h1 = bf16_bits_rn(v1);
        const uint32_t l0 = bf16_bits_rn(__fsub_rn(v0, __uint_as_float(h0 << 16)));
        const uint32_t l1 = bf16_bits_rn(__fsub_rn(v1, __uint_as_float(h1 << 16)));
        hi2 = h0 | (h1 << 16);
        lo2 = l0 | (l1 << 16);
    } else {
        const float h0 = veltkamp_hi11(v0), h1 = veltkamp_hi11(v1);
        hi2 = pack_f16x2(h0, h1);
        lo2 = pack_f16x2(__fsub_rn(v0, h0), __fsub_rn(v1, h1));
    }
}

// an integer-valued pair (|n| <= 256: exact in both formats), packed
template <bool BF16>
__device__ __forceinline__ uint32_t pack_int2(float n0, float n1) {
    if (BF16) return (__float_as_uint(n0) >> 16) | (__float_as_uint(n1) & 0xFFFF0000u);
    return pack_f16x2(n0, n1);
}

// the same pair split through the format-conversion unit (round to nearest even twice)
template <bool BF16>
__device__ __forceinline__ void split2_cvt(float v0, float v1, uint32_t& hi2, uint32_t& lo2) {
    uint16_t h[2], l[2];
    const float v[2] = {v0, v1};
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        if (BF16) {
            const __nv_bfloat16 x = __float2bfloat16_rn(v[t]);
            h[t] = __bfloat16_as_ushort(x);
            l[t] = __bfloat16_as_ushort(__float2bfloat16_rn(v[t] - __bfloat162float(x)));
        } else {
            const __half x = __float2half_rn(v[t]);
            h[t] = __half_as_ushort(x);
            l[t] = __half_as_ushort(__float2half_rn(v[t] - __half2float(x)));
        }
    }
    hi2 = (uint32_t)h[0] | ((uint32_t)h[1] << 16);
    lo2 = (uint32_t)l[0] | ((uint32_t)l[1] << 16);
}

// 8 consecutive K elements of row r of a K-major tile with K columns: one 16-byte row of a
// core matrix in each of the hi and lo tiles.  CVT: split through the conversion unit (the
// whitening pass, H2, measured faster that way; the other passes measured faster without).
template <bool BF16, bool CVT = false>
__device__ __forceinline__ bool store8_split(uint16_t* thi, uint16_t* tlo, int r, int k0, int K,
                                             const float v[8]) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (CVT) split2_cvt<BF16>(v[2 * q], v[2 * q + 1], h[q], l[q]);
        else split2<BF16>(v[2 * q], v[2 * q + 1], h[q], l[q]);
    }
    const uint32_t off = tc::kmajor_offset(r, k0, K) >> 1;  // in 16-bit elements
    *reinterpret_cast<uint4*>(thi + off) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(tlo + off) = make_uint4(l[0], l[1], l[2], l[3]);
    return ((l[0] | l[1] | l[2] | l[3]) & 0x7FFF7FFFu) != 0u;  // a low half other than +-0
}

// 8 consecutive K values of row r, split into the integer part n = rint(v) (exact in both
// 16-bit formats for |n| <= 256) and the fraction f = v - n as a high and a low 16-bit half
template <bool BF16>
__device__ __forceinline__ bool store8_int_frac(uint16_t* tn, uint16_t* tfh, uint16_t* tfl, int r,
                                                int k0, int K, const float v[8]) {
    uint32_t n[4], fh[4], fl[4];
    constexpr float kRnd = 12582912.0f;  // 1.5 * 2^23: x + kRnd - kRnd rounds to an integer (RN)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const float x0 = v[2 * q], x1 = v[2 * q + 1];
        const float n0 = __fsub_rn(__fadd_rn(x0, kRnd), kRnd), n1 = __fsub_rn(__fadd_rn(x1, kRnd), kRnd);
        n[q] = pack_int2<BF16>(n0, n1);
        split2<BF16>(__fsub_rn(x0, n0), __fsub_rn(x1, n1), fh[q], fl[q]);
    }
    const uint32_t off = tc::kmajor_offset(r, k0, K) >> 1;
    *reinterpret_cast<uint4*>(tn + off) = make_uint4(n[0], n[1], n[2], n[3]);
    *reinterpret_cast<uint4*>(tfh + off) = make_uint4(fh[0], fh[1], fh[2], fh[3]);
    *reinterpret_cast<uint4*>(tfl + off) = make_uint4(fl[0], fl[1], fl[2], fl[3]);
    return ((fh[0] | fh[1] | fh[2] | fh[3] | fl[0] | fl[1] | fl[2] | fl[3]) & 0x7FFF7FFFu) != 0u;
}

// Operand tiles of the tensor-core passes in the 64 KB region h.mx (byte offsets), two
// buffers per pass: the MMAs of one chunk run while the next chunk is staged.  The MMAs
// are M = 64 (A rows), N = 32 or 48 (B rows): the tensor cores read their operands from
// shared memory for every MMA, and that traffic (not the arithmetic) sets their time, so
// the shapes stay as close to the live rows as the instruction allows.  A tile holds only
// its live rows (K-major, no swizzle: 8-row groups of K/8 core matrices, 128 B each).  An
// A descriptor reads 64 rows from the tile start; the rows past a shorter tile hold other
// data of the region and only produce rows of D that are never read.  Every such read
// window ends inside the region.
namespace tl {
constexpr uint32_t kRegion = 65536;
constexpr uint32_t kWinK64 = 64 * 64 * 2;  // bytes an M = 64, K = 64 A descriptor reads
constexpr uint32_t kWinK32 = 64 * 32 * 2;  // M = 64, K = 32
// H1, K = 64: integer part, fraction high and low halves (48 rows: features, the constant
// in row 36); then the int32 sums
constexpr uint32_t kH1Tile = 48 * 64 * 2, kH1Buf = 3 * kH1Tile, kH1Sums = 49152;
constexpr uint32_t kH1SumsBytes = 36 * 40 * 4;
// H2: see H2L below (its layout depends on the candidates per tile)
// H3, K = 64: A = weights (32 rows: beta) high / low; B = Z' (48 rows) high / low
constexpr uint32_t kH3W = 4096, kH3WBuf = 2 * kH3W, kH3Z = 16384, kH3ZTile = 6144, kH3ZBuf = 2 * kH3ZTile;
static_assert(kH1Buf + 2 * kH1Tile + kWinK64 <= kRegion && 2 * kH1Buf <= kH1Sums &&
                  kH1Sums + kH1SumsBytes <= kRegion, "H1 tiles");
static_assert(kH3WBuf + kH3W + kWinK64 <= kRegion && 2 * kH3WBuf <= kH3Z && kH3Z + 2 * kH3ZBuf <= kRegion,
              "H3 tiles");
}  // namespace tl

__device__ __forceinline__ uint16_t* tile(Hql& h, uint32_t byte_off) { return h.mx + (byte_off >> 1); }

__device__ __forceinline__ void zero_region(Hql& h, uint32_t off, uint32_t bytes) {
    uint4* p = reinterpret_cast<uint4*>(tile(h, off));
    for (int i = threadIdx.x; i < (int)(bytes / 16); i += kThreads) p[i] = make_uint4(0, 0, 0, 0);
}

// D (+)= A * B^T over K columns with split operands (issued by one thread)
__device__ __forceinline__ void mma3(uint32_t tmem, const uint16_t* ahi, const uint16_t* alo,
                                     const uint16_t* bhi, const uint16_t* blo, int K, uint32_t idesc,
                                     bool accumulate) {
    const uint32_t sbo = (uint32_t)(K / 8) * 128u;
    const uint32_t a0 = tc::smem_addr(ahi), a1 = tc::smem_addr(alo);
    const uint32_t b0 = tc::smem_addr(bhi), b1 = tc::smem_addr(blo);
    for (int kk = 0; kk < K / 16; ++kk) {
        const uint32_t o = (uint32_t)kk * 256u;
        tc::mma_f16(tmem, tc::smem_desc(a0 + o, 128, sbo), tc::smem_desc(b0 + o, 128, sbo), idesc,
                    accumulate || kk > 0);
        tc::mma_f16(tmem, tc::smem_desc(a0 + o, 128, sbo), tc::smem_desc(b1 + o, 128, sbo), idesc, true);
        tc::mma_f16(tmem, tc::smem_desc(a1 + o, 128, sbo), tc::smem_desc(b0 + o, 128, sbo), idesc, true);
    }
}

// The chunk pipeline of a pass: [tiles_ready] issue the MMAs of chunk c, stage chunk c + 1
// into the other buffer, [mma_wait] chunk c complete.  Issuing an MMA stalls the issuing
// thread until the tensor core takes it; the issuer is lane 0 of the last warp, whose
// threads take one Z' staging task each (the second round of Z' tasks goes to the first
// two warps).
constexpr int kIssuer = kThreads - 32;
// Staged tiles visible to the tensor cores; every thread past the previous chunk's
// tensor-memory reads.
__device__ __forceinline__ void tiles_ready() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
}

// the same, returning whether any thread's flag is set (a CTA-uniform value)
__device__ __forceinline__ bool tiles_ready_or(bool flag) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc::fence_before();
    const bool any = __syncthreads_or(flag ? 1 : 0) != 0;
    tc::fence_after();
    return any;
}

template <typename IssueF>
__device__ __forceinline__ void mma_issue(Smem& sm, IssueF issue) {
    if (threadIdx.x == kIssuer) {
        issue();
        tc::mma_commit(&sm.mma_bar);
    }
}

__device__ __forceinline__ void mma_wait(Smem& sm, uint32_t& mph) {
    if (!tc::mbar_wait(&sm.mma_bar, mph, 1u << 26)) atomicExch(&sm.mma_err, 1);
    mph ^= 1u;
    tc::fence_after();
}

// stage rows 0..36 of Z^T for candidates [c0, c0+n): z' (feature rows 0..35, zero beyond
// nz) and the constant one (row 36)
// Returns whether this thread staged a value that one 16-bit part does not hold exactly (a
// non-zero fraction, INTFRAC; a non-zero low half, otherwise).
template <bool BF16, bool INTFRAC, int CH>
__device__ __forceinline__ bool stage_zt(Smem& sm, int c0, int n, int nz, float shift, uint16_t* t0,
                                         uint16_t* t1, uint16_t* t2) {
    Hql& h = sm.hql;
    // live rows: the nz = 4 + Ny features and the constant (row 36); the other rows stay
    // at the zeros the pass started from.  Row slot ri < nz is feature ri, slot nz the
    // constant.  A quarter-warp writes one 16-byte column group of 8 consecutive slots
    // (one 128-byte core matrix: no bank conflicts); one task per thread for nz <= 31.
    // The second round of tasks (rows 32..36) goes to the first two warps, with the lanes
    // of each 8-lane group in reverse order: the live ones (rows 32..36) then fall on lanes
    // 3..7 of the group, where the beta pass with the default 25-value grid gives them no
    // weight row (h3_mixed).
    // (CH candidates per chunk: CH / 8 column groups; tasks of a row group: 8 rows x CH / 8)
    const int nr = nz + 1;
    const int ntask = ((nr + 7) >> 3) * CH;  // nz <= 36: at most 5 row groups, 5 CH tasks
    bool inexact = false;
    for (int rnd = 0; rnd < 2; ++rnd) {
        const int idx = rnd == 0 ? (int)threadIdx.x : kThreads + ((int)threadIdx.x ^ 7);
        if (idx >= ntask) continue;
        const int ri = ((idx / CH) << 3) | (idx & 7), g8 = (idx % CH) >> 3;
        if (ri >= nr) continue;
        const int a = ri < nz ? ri : 36;
        const int ka = a < kZs ? h.koff[a] : -1;
        // the group's 8 candidate indices in one 16-byte load (c0 + 8 g8 is a multiple of 8;
        // h.cand holds 7 entries past the last candidate, so a group past M reads inside it)
        const uint4 cq = *reinterpret_cast<const uint4*>(&h.cand[c0 + 8 * g8]);
        const uint32_t cw[4] = {cq.x, cq.y, cq.z, cq.w};
        float v[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const int j = 8 * g8 + t;
            float x = 0.0f;
            if (j < n) {
                if (a == 36) x = 1.0f;
                else if (ka >= 0) x = sm.S[(int)((cw[t >> 1] >> (16 * (t & 1))) & 0xFFFFu) + ka] - shift;
            }
            v[t] = x;
        }
        if (INTFRAC) inexact |= store8_int_frac<BF16>(t0, t1, t2, a, 8 * g8, CH, v);
        else inexact |= store8_split<BF16>(t0, t1, a, 8 * g8, CH, v);
    }
    return inexact;
}

// H1 on tensor cores: D[a][b] = sum_j z'_ja z'_jb and D[a][36] = sum_j z'_ja, with
// z' = n + f (integer part n, fraction f = fh + fl).  The integer products n_a n_b are
// exact in 16 bits and their sum over 4 chunks (256 candidates, |n| <= 255: at most
// 16,646,400) stays below 2^24, so the FP32 accumulator holds it exactly; it is read out
// every 4 chunks into int32.  The fractional terms n f^T + f n^T + fh fh^T are symmetric
// in pairs: X = n (fh + fl)^T (tensor memory columns 64..111) and Y = fh fh^T (columns
// 128..175) accumulate in FP32, and the readout forms X + X^T + Y.  The same integer /
// fraction split as the CUDA-core path, so the covariance keeps its precision through the
// cancellation in Eq. (8).  Row 36 of the tiles is the constant one (n = 1, f = 0), so
// column 36 of the integer sums holds sum_j n_a and (X + X^T)[a][36] holds sum_j f_a.
// CH: candidates per chunk (32 or 64: the MMAs' K); the products are accumulated over the
// same 16-candidate slices in the same order whatever CH, so the result does not depend on it.
template <bool BF16, int CH>
__device__ __noinline__ void h1_mixed(int M, int nz, float shift, uint32_t tmem, uint32_t mph) {
    static_assert(CH == 32 || CH == 64, "H1 chunk");
    constexpr int kRead = 256 / CH;  // chunks between integer readouts (256 candidates)
    Smem& sm = smem_ref();
    Hql& h = sm.hql;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int nchunks = (M + CH - 1) / CH;
    const uint32_t idesc = tc::idesc_f16(64, 48, BF16);
    __syncthreads();  // the tiles share storage with buffers of the previous phase
    // both buffers (rows past the live features stay zero) and the integer sums
    zero_region(h, 0, 2 * tl::kH1Buf);
    zero_region(h, tl::kH1Sums, tl::kH1SumsBytes);
    __syncthreads();
    // warps 0..2, lanes 0..15: row arow of D (M = 64 layout), for arow <= 36
    const int arow = 16 * wid + lane;
    const bool reader = wid < 3 && lane < 16 && arow < 37;
    const uint32_t tlane = (uint32_t)(32 * wid) << 16;
    // integer sums: the thread's own row of an int32 array past the tiles (p1 shares
    // storage with the tiles)
    int(*nacc)[40] = reinterpret_cast<int(*)[40]>(tile(h, tl::kH1Sums));
    auto tb = [&](int b, int t) { return tile(h, (uint32_t)b * tl::kH1Buf + (uint32_t)t * tl::kH1Tile); };
    // A chunk whose staged values are all integers (candidates made of received pixels only)
    // has zero fractions: its X and Y products are left out.  xy_live: some chunk issued
    // them (X and Y hold sums).
    bool fr = stage_zt<BF16, true, CH>(sm, 0, min(CH, M), nz, shift, tb(0, 0), tb(0, 1), tb(0, 2));
    bool xy_live = false;
    for (int ch = 0; ch < nchunks; ++ch) {
        const int b = ch & 1;
        const bool frac = tiles_ready_or(fr);
        const bool xy_acc = xy_live;
        mma_issue(sm, [&]() {
            const uint32_t sbo = (CH / 8) * 128;
            const uint32_t an = tc::smem_addr(tb(b, 0)), ah = tc::smem_addr(tb(b, 1)),
                           al = tc::smem_addr(tb(b, 2));
            for (int kk = 0; kk < CH / 16; ++kk) {
                const uint32_t o = (uint32_t)kk * 256u;
                const uint64_t dn = tc::smem_desc(an + o, 128, sbo), dh = tc::smem_desc(ah + o, 128, sbo),
                               dl = tc::smem_desc(al + o, 128, sbo);
                tc::mma_f16(tmem, dn, dn, idesc, (ch % kRead) != 0 || kk > 0);  // integer part: 256 candidates
                if (frac) {
                    tc::mma_f16(tmem + 64, dn, dh, idesc, xy_acc || kk > 0);   // X = n (fh + fl)^T
                    tc::mma_f16(tmem + 64, dn, dl, idesc, true);
                    tc::mma_f16(tmem + 128, dh, dh, idesc, xy_acc || kk > 0);  // Y = fh fh^T
                }
            }
            sm.st[ST_MMA_FLOPS] += (frac ? 4ull : 1ull) * (CH / 16) * (2ull * 64 * 48 * 16);
        });
        xy_live = xy_live || frac;
        if (ch + 1 < nchunks) {  // the next chunk, while these MMAs run
            const int c1 = (ch + 1) * CH;
            fr = stage_zt<BF16, true, CH>(sm, c1, min(CH, M - c1), nz, shift, tb(b ^ 1, 0), tb(b ^ 1, 1),
                                          tb(b ^ 1, 2));
        }
        mma_wait(sm, mph);
        if (wid < 3 && ((ch % kRead) == kRead - 1 || ch == nchunks - 1)) {  // exact sums into int32
            for (int c = 0; c < 5; ++c) {  // columns 0..39 in groups of 8 (36: column sums)
                float D[8];
                tc::tmem_ld8(tmem + tlane + 8 * c, D);
                if (reader && arow < 36) {
#pragma unroll
                    for (int t = 0; t < 8; ++t) nacc[arow][8 * c + t] += __float2int_rn(D[t]);
                }
            }
        }
        // (the next chunk's tiles_ready orders these tensor-memory reads before its MMAs)
    }
    // every MMA has completed: the operand tiles are dead.  X goes to a scratch array at
    // the start of the region (p1 and the integer sums lie past it), X + Y to the row of
    // cfrac; then cfrac += X^T.
    float(*xs)[40] = reinterpret_cast<float(*)[40]>(tile(h, 0));
    static_assert(37 * 40 * sizeof(float) <= 2 * tl::kH1Buf, "X scratch inside the tiles");
    if (wid < 3) {
        for (int c = 0; c < 5; ++c) {
            float X[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, Y[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            if (xy_live) {  // (CTA-uniform)
                tc::tmem_ld8(tmem + tlane + 64 + 8 * c, X);
                tc::tmem_ld8(tmem + tlane + 128 + 8 * c, Y);
            }
            if (reader) {
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const int b = 8 * c + t;
                    xs[arow][b] = X[t];
                    if (arow < 36 && b < 37) {
                        if (b < 36) {
                            h.p1.cfrac[arow][b] = X[t] + Y[t];
                            h.p1.cint[arow][b] = nacc[arow][b];
                        } else {
                            h.colF[arow] = X[t] + Y[t];
                            h.colNi[arow] = nacc[arow][36];
                        }
                    }
                }
            }
        }
    }
    __syncthreads();
    for (int idx = tid; idx < 36 * 37; idx += kThreads) {
        const int a = idx / 37, b = idx - a * 37;
        if (b < 36) h.p1.cfrac[a][b] += xs[b][a];
        else h.colF[a] += xs[36][a];
    }
    tc::fence_before();
    __syncthreads();
}

// H2 on tensor cores: u_j = L^-1 (y_j - y0) for CH candidates at a time (CH = 64: MMA
// M = 64; CH = 128: M = 128), d_j = ||u_j||^2; u_j goes to ubuf (row j, 32 floats) for the
// leave-one-out pass.  Each candidate's row is an independent product, so the result does not
// depend on CH.  Layout of the region: A buffers (CH rows x K = 32, high and low halves, two
// buffers), B = L^-1 (32 rows, high and low), then the staging rows of u (CH x 128 bytes).
template <int CH>
struct H2L {
    static constexpr uint32_t kA = CH * 64, kABuf = 2 * kA, kB = 2 * kABuf, kBTile = 2048, kU = kB + 2 * kBTile;
    static_assert(kU + CH * 128 <= tl::kRegion, "H2 tiles");
};

template <bool BF16, int CH>
__device__ __noinline__ float h2_mixed(int M, int ny, float shift, uint32_t tmem, uint32_t mph,
                                       float* ubuf) {
    static_assert(CH == 64 || CH == 128, "H2 chunk");
    using L = H2L<CH>;
    constexpr int kRowsW = CH / 4;  // accumulator rows per reading warp (warps 0..3)
    // live coordinates: groups of 8 tensor-memory columns and of 4 stored floats (past Ny the
    // whitened coordinates are exact zeros)
    const int n8 = (ny + 7) >> 3, nq = (ny + 3) >> 2;
    // K = N = 16 when Ny <= 16: the dropped K slices and output columns hold exact zeros, so
    // the products are the same bit for bit, at half the MMAs and operand staging
    const int KH = ny <= 16 ? 16 : 32, G = KH >> 3, gsh = KH == 16 ? 4 : 5;
    Smem& sm = smem_ref();
    Hql& h = sm.hql;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int nchunks = (M + CH - 1) / CH;
    __syncthreads();  // the tiles share storage with buffers of the previous phase
    // B = L^-1 (KH rows k x KH columns l), staged once
    uint16_t* bhi = tile(h, L::kB);
    uint16_t* blo = tile(h, L::kB + L::kBTile);
    if (tid < KH * G) {
        const int k = (tid & 7) | ((tid >> gsh) << 3), l8 = (tid >> 3) & (G - 1);  // conflict-free stores
        float v[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) v[t] = h.Linv[k][8 * l8 + t];
        store8_split<BF16, true>(bhi, blo, k, 8 * l8, KH, v);
    }
    // A = E (rows: candidates, columns: context) of chunk ch into buffer ch & 1: CH rows x G
    // column groups; a quarter-warp stores 8 consecutive rows of one column group
    // (conflict-free)
    auto stage_a = [&](int ch) {
        const int c0 = ch * CH, n = min(CH, M - c0);
        const uint32_t o = (uint32_t)(ch & 1) * L::kABuf;
        for (int q = tid; q < G * CH; q += kThreads) {
            const int j = (q & 7) | ((q >> gsh) << 3), l8 = (q >> 3) & (G - 1);
            float v[8];
            const int base = j < n ? h.cand[c0 + j] : 0;
            // the 8 context offsets and centred context values of column group l8 in 16-byte
            // loads (l8 < 4: inside the 36-entry lists)
            const uint4 oq = *reinterpret_cast<const uint4*>(&h.off[8 * l8]);
            const float4 y0v = *reinterpret_cast<const float4*>(&h.ys[8 * l8]);
            const float4 y1v = *reinterpret_cast<const float4*>(&h.ys[8 * l8 + 4]);
            const uint32_t ow[4] = {oq.x, oq.y, oq.z, oq.w};
            const float yv[8] = {y0v.x, y0v.y, y0v.z, y0v.w, y1v.x, y1v.y, y1v.z, y1v.w};
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const int l = 8 * l8 + t;
                const int o = (int)(short)((ow[t >> 1] >> (16 * (t & 1))) & 0xFFFFu);
                v[t] = (j < n && l < ny) ? (sm.S[base + o] - shift) - yv[t] : 0.0f;
            }
            store8_split<BF16, true>(tile(h, o), tile(h, o + L::kA), j, 8 * l8, KH, v);
        }
    };
    // d_j = ||u_j||^2 of chunk ch from tensor-memory columns 32 (ch & 1) .. +31.  Candidate
    // j of the chunk: M = 64, lane 16w + j%16 of warp w = j / 16; M = 128, lane j%32 of warp
    // w = j / 32.
    float lmin = INFINITY;
    auto read_d = [&](int ch) {
        if (wid < 4) {
            const int c0 = ch * CH, n = min(CH, M - c0), j = kRowsW * wid + lane;
            const bool row_lane = kRowsW == 32 || lane < 16;
            // the warp's rows of u pass through shared memory, so that the global stores are
            // whole 128-byte rows (8 lanes per row; a bulk copy through the async proxy
            // measured slower: its proxy fence waits behind the MMAs in flight)
            float* us = reinterpret_cast<float*>(tile(h, L::kU)) + kRowsW * 32 * wid;
            float dd = 0.0f;
            for (int c = 0; c < n8; ++c) {  // live groups of 8 columns (few live registers)
                float u[8];
                tc::tmem_ld8(tmem + ((uint32_t)(32 * wid) << 16) + 32 * (ch & 1) + 8 * c, u);
#pragma unroll
                for (int k = 0; k < 8; ++k) dd = __fmaf_rn(u[k], u[k], dd);
                if (row_lane) {
                    float* row = us + 32 * lane;
                    *reinterpret_cast<float4*>(row + ubuf_pos(lane, 2 * c)) = make_float4(u[0], u[1], u[2], u[3]);
                    *reinterpret_cast<float4*>(row + ubuf_pos(lane, 2 * c + 1)) = make_float4(u[4], u[5], u[6], u[7]);
                }
            }
            __syncwarp();
#pragma unroll
            for (int t = 0; t < kRowsW / 4; ++t) {  // rows x 8 float4, 4 rows per instruction
                const int idx = lane + 32 * t, r = idx >> 3, p4 = idx & 7;  // p4: physical position
                const int c4 = p4 ^ (r & 7);                                 // its logical group
                if (kRowsW * wid + r < n && c4 < nq)
                    *reinterpret_cast<float4*>(ubuf + (size_t)(c0 + kRowsW * wid + r) * kMaxNy + 4 * p4) =
                        *reinterpret_cast<const float4*>(us + 32 * r + 4 * p4);
            }
            __syncwarp();  // the staging rows take the next chunk
            if (row_lane && j < n) {
                h.d[c0 + j] = dd;
                lmin = fminf(lmin, dd);
            }
        }
    };
    stage_a(0);
    for (int ch = 0; ch < nchunks; ++ch) {
        const uint32_t o = (uint32_t)(ch & 1) * L::kABuf;
        tiles_ready();
        mma_issue(sm, [&]() {
            mma3(tmem + 32 * (ch & 1), tile(h, o), tile(h, o + L::kA), bhi, blo, KH,
                 tc::idesc_f16(CH, KH, BF16), false);
            sm.st[ST_MMA_FLOPS] += 3ull * (KH / 16) * (2ull * CH * KH * 16);
        });
        if (ch + 1 < nchunks) stage_a(ch + 1);  // while the MMAs of chunk ch run
        if (ch > 0) read_d(ch - 1);            // (the other tensor-memory columns)
        mma_wait(sm, mph);
    }
    read_d(nchunks - 1);
    tc::fence_before();
    __syncthreads();  // tensor memory read before the next pass's MMAs
    return lmin;
}

// H3 on tensor cores: D[b][k] = sum_j w_j(b) z'_j[k] with w_j(b) = exp(-(d_j - dmin)/(2 beta_b))
template <bool BF16>
__device__ __noinline__ void h3_mixed(const KParams& P, int M, int nz, float shift, float dmin,
                                         uint32_t tmem, uint32_t mph) {
    Smem& sm = smem_ref();
    Hql& h = sm.hql;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int nchunks = (M + kCh - 1) / kCh;
    const int nb = P.nbeta;
    __syncthreads();  // the tiles share storage with buffers of the previous phase
    zero_region(h, tl::kH3Z, 2 * tl::kH3ZBuf);  // Z' rows past the live features stay zero
    __syncthreads();
    auto zt = [&](int b, int t) { return tile(h, tl::kH3Z + (uint32_t)b * tl::kH3ZBuf + (uint32_t)t * tl::kH3ZTile); };
    auto wt = [&](int b, int t) { return tile(h, (uint32_t)b * tl::kH3WBuf + (uint32_t)t * tl::kH3W); };
    auto stage = [&](int ch) {
        const int c0 = ch * kCh, n = min(kCh, M - c0), bf = ch & 1;
        stage_zt<BF16, false, kCh>(sm, c0, n, nz, shift, zt(bf, 0), zt(bf, 1), nullptr);
        // A = W (rows: beta, columns: candidates), 32 rows x 8 column groups; a quarter-warp
        // stores 8 consecutive rows of one column group (conflict-free)
        {  // one task per thread; rows 24..31 (of which only 24 is live with the default
           // 25-value grid) go to the first two warps, which take the second round of Z'
           // tasks on other lanes (stage_zt), so that no thread stages three rows
            const int q = tid;
            const int b = (q & 7) | (((q >> 6) ^ 3) << 3), g8 = (q >> 3) & 7;
            if (b < nb) {
                float v[8];
                const float ib = P.inv2beta[b];
                // the group's 8 distances in two 16-byte loads (h.d holds 7 entries past the
                // last candidate)
                const float4 d0 = *reinterpret_cast<const float4*>(&h.d[c0 + 8 * g8]);
                const float4 d1 = *reinterpret_cast<const float4*>(&h.d[c0 + 8 * g8 + 4]);
                const float dv[8] = {d0.x, d0.y, d0.z, d0.w, d1.x, d1.y, d1.z, d1.w};
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const int j = 8 * g8 + t;
                    v[t] = j < n ? __expf(-(dv[t] - dmin) * ib) : 0.0f;
                }
                store8_split<BF16>(wt(bf, 0), wt(bf, 1), b, 8 * g8, 64, v);
            }
        }
    };
    stage(0);
    for (int ch = 0; ch < nchunks; ++ch) {
        const int bf = ch & 1;
        tiles_ready();
        mma_issue(sm, [&]() {
            mma3(tmem, wt(bf, 0), wt(bf, 1), zt(bf, 0), zt(bf, 1), 64, tc::idesc_f16(64, 48, BF16), ch > 0);
            sm.st[ST_MMA_FLOPS] += 12ull * (2ull * 64 * 48 * 16);
        });
        if (ch + 1 < nchunks) stage(ch + 1);  // while the MMAs of chunk ch run
        mma_wait(sm, mph);
    }
    if (wid < 2) {  // beta b in lane 16w + b%16 of warp w = b / 16 (M = 64 layout)
        const int b = 16 * wid + lane;
        for (int c = 0; c < 5; ++c) {  // columns 0..39 in groups of 8
            float D[8];
            tc::tmem_ld8(tmem + ((uint32_t)(32 * wid) << 16) + 8 * c, D);
            if (lane < 16 && b < nb) {
#pragma unroll
                for (int t = 0; t < 8; ++t)
                    if (8 * c + t < 37) h.accBd[b][8 * c + t] = df_make(D[t]);
            }
        }
    }
    tc::fence_before();
    __syncthreads();
}

// IDL distances of every candidate window on tensor cores (mixed precision, option
// SKMMSE_FLAG_IDL_TC): for the rings after the first, the distances of Eq. (15) of all
// 43 x 43 window positions in one pass.  With S' = S - cen, y0' = y0 - cen and m the context
// mask of the 6x6 window,
//   d[u][v] = sum_{r,c} m[r][c] (S'[u+r][v+c] - y0'[r][c])^2
//           = sum_r sum_x S'[u+r][x] (-2 T[r][x-v]) + S'[u+r][x]^2 M[r][x-v]  +  sum m y0'^2,
// T = m y0', M = m (zero outside 0 <= x-v <= 5): for each window row r a Toeplitz product
// A_r B_r^T with A_r[u][x] = S'[u+r][x] (u: M = 64 rows, 43 live; x: K = 48) and B_r[v][x]
// (v: N = 48 rows, 43 live).  S' and T are split into high and low 16-bit halves (three
// MMAs), S'^2 too (two MMAs against the exact 0/1 mask); all accumulate in one FP32
// tensor-memory tile.  Integer contexts and windows (received pixels) are exact in both
// formats.  d goes to h.d[u * 43 + v].
namespace tli {
constexpr uint32_t kA = 64 * 48 * 2, kB = 48 * 48 * 2;  // tile bytes
constexpr uint32_t kAhi = 0, kAlo = kA, kQhi = 2 * kA, kQlo = 3 * kA, kBhi = 4 * kA, kBlo = 4 * kA + kB,
                   kMk = 4 * kA + 2 * kB, kEnd = 4 * kA + 3 * kB;
static_assert(kEnd <= tl::kRegion && kBhi % 128 == 0 && kBlo % 128 == 0 && kMk % 128 == 0, "IDL tiles");
}  // namespace tli

template <bool BF16>
__device__ __noinline__ void idl_tc_distances(int wr, int wc, unsigned long long ymask, float cen,
                                              uint32_t tmem, uint32_t mph) {
    Smem& sm = smem_ref();
    Hql& h = sm.hql;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const uint32_t idesc = tc::idesc_f16(64, 48, BF16);
    float y2 = 0.0f;  // sum m y0'^2 (every thread, the same order)
#pragma unroll
    for (int k = 0; k < 36; ++k)
        if ((ymask >> k) & 1ull) {
            const float t = sm.S[(wr + k / 6) * kReg + wc + k % 6] - cen;
            y2 = __fmaf_rn(t, t, y2);
        }
    __syncthreads();  // the tiles share storage with the IDL slots' neighbours of the union
    for (int r = 0; r < 6; ++r) {
        // A rows u (64 x 6 column groups) and B rows v (48 x 6 column groups); a quarter-warp
        // stores 8 consecutive rows of one column group (conflict-free)
        for (int q = tid; q < 64 * 6 + 48 * 6; q += kThreads) {
            const bool isA = q < 64 * 6;
            const int qq = isA ? q : q - 64 * 6;
            const int row = (qq & 7) | ((qq / 48) << 3), g = (qq >> 3) % 6;
            float v[8];
            if (isA) {
                const int sr = row + r;
                float v2[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const float x = (row < kNpos && sr < kReg) ? sm.S[sr * kReg + 8 * g + t] - cen : 0.0f;
                    v[t] = x;
                    v2[t] = __fmul_rn(x, x);
                }
                store8_split<BF16>(tile(h, tli::kAhi), tile(h, tli::kAlo), row, 8 * g, 48, v);
                store8_split<BF16>(tile(h, tli::kQhi), tile(h, tli::kQlo), row, 8 * g, 48, v2);
            } else {
                float mk[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const int c = 8 * g + t - row;  // window column of x = 8g + t for v = row
                    const bool on = row < kNpos && c >= 0 && c < 6 && ((ymask >> (6 * r + c)) & 1ull);
                    v[t] = on ? -2.0f * (sm.S[(wr + r) * kReg + wc + c] - cen) : 0.0f;
                    mk[t] = on ? 1.0f : 0.0f;
                }
                store8_split<BF16>(tile(h, tli::kBhi), tile(h, tli::kBlo), row, 8 * g, 48, v);
                uint32_t w[4];
#pragma unroll
                for (int p2 = 0; p2 < 4; ++p2) w[p2] = pack_int2<BF16>(mk[2 * p2], mk[2 * p2 + 1]);
                const uint32_t off = tc::kmajor_offset(row, 8 * g, 48) >> 1;
                *reinterpret_cast<uint4*>(tile(h, tli::kMk) + off) = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
        tiles_ready();
        mma_issue(sm, [&]() {
            mma3(tmem, tile(h, tli::kAhi), tile(h, tli::kAlo), tile(h, tli::kBhi), tile(h, tli::kBlo), 48, idesc,
                 r > 0);
            const uint32_t sbo = (48 / 8) * 128;
            const uint32_t q0 = tc::smem_addr(tile(h, tli::kQhi)), q1 = tc::smem_addr(tile(h, tli::kQlo));
            const uint32_t bm = tc::smem_addr(tile(h, tli::kMk));
            for (int kk = 0; kk < 3; ++kk) {
                const uint32_t o = (uint32_t)kk * 256u;
                const uint64_t dm = tc::smem_desc(bm + o, 128, sbo);
                tc::mma_f16(tmem, tc::smem_desc(q0 + o, 128, sbo), dm, idesc, true);
                tc::mma_f16(tmem, tc::smem_desc(q1 + o, 128, sbo), dm, idesc, true);
            }
            sm.st[ST_MMA_FLOPS] += 15ull * (2ull * 64 * 48 * 16);
        });
        mma_wait(sm, mph);  // (the tiles take the next row)
    }
    // d of row u from tensor-memory lane 32 (u / 16) + u % 16 (M = 64 layout)
    if (wid < 4) {
        const int u = 16 * wid + lane;
        for (int c = 0; c < 6; ++c) {
            float D[8];
            tc::tmem_ld8(tmem + ((uint32_t)(32 * wid) << 16) + 8 * c, D);
            if (lane < 16 && u < kNpos) {
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const int v = 8 * c + t;
                    if (v < kNpos) h.d[u * kNpos + v] = fmaxf(D[t] + y2, 0.0f);
                }
            }
        }
    }
    tc::fence_before();
    __syncthreads();
}

// packed two-lane FP32 (sm_100+): each lane an IEEE round-to-nearest operation
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 f2_pack(float a, float b) {
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void f2_unpack(f32x2 v, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f32x2 f2_sub(f32x2 a, f32x2 b) {
    f32x2 r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f32x2 f2_fma(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// one step of a max-subtracted online softmax sum: score sc, values [x' | G u]
// The rescale is a select, not a branch (the lanes are different members and diverge): the
// factor is exp(m - sc) for a new maximum (0 when m = -inf) and exactly 1 otherwise.  Its
// products are rounded on their own (__fmul_rn: not fused with the additions that follow),
// so the sums are those of the branch bit for bit.
__device__ __forceinline__ void h5_online(float sc, float4 xv, float4 gv, float& m, float& sw, float sa[8]) {
    const float e = __expf(m - sc);
    const float r = sc > m ? e : 1.0f;
    sw = __fmul_rn(sw, r);
#pragma unroll
    for (int k = 0; k < 8; ++k) sa[k] = __fmul_rn(sa[k], r);
    m = fmaxf(m, sc);
    const float w = __expf(sc - m);
    sw += w;
    sa[0] = __fmaf_rn(w, xv.x, sa[0]);
    sa[1] = __fmaf_rn(w, xv.y, sa[1]);
    sa[2] = __fmaf_rn(w, xv.z, sa[2]);
    sa[3] = __fmaf_rn(w, xv.w, sa[3]);
    sa[4] = __fmaf_rn(w, gv.x, sa[4]);
    sa[5] = __fmaf_rn(w, gv.y, sa[5]);
    sa[6] = __fmaf_rn(w, gv.z, sa[6]);
    sa[7] = __fmaf_rn(w, gv.w, sa[7]);
}

// member mode of the leave-one-out pass for one buffered group of nc candidates: the
// squared whitened distance of member u (its first NQ coordinate groups; the rest are
// zero) to each candidate, in packed two-lane FP32, and the online sums; cself is the
// member's own index in the group (skipped), or out of range
template <int NQ>
__device__ __forceinline__ void h5_members(const float (*wb)[kWb], const float* ui, int nc, int cself,
                                           float ib, float& m, float& sw, float sa[8]) {
    f32x2 U[2 * NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(&ui[4 * q]);
        U[2 * q] = v.x;
        U[2 * q + 1] = v.y;
    }
    for (int c = 0; c < nc; ++c) {
        f32x2 d2 = 0ull;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(&wb[c][12 + 4 * q]);
            f32x2 t = f2_sub(U[2 * q], v.x);
            d2 = f2_fma(t, t, d2);
            t = f2_sub(U[2 * q + 1], v.y);
            d2 = f2_fma(t, t, d2);
        }
        if (c == cself) continue;
        float dl, dh;
        f2_unpack(d2, dl, dh);
        h5_online(-(dl + dh) * ib, *reinterpret_cast<const float4*>(&wb[c][0]),
                  *reinterpret_cast<const float4*>(&wb[c][4]), m, sw, sa);
    }
}

// Not inlined: HQL runs for a small share of the patches, and as a function of its own its
// register demand does not spill the per-step loop of the kernel.
// The arguments are scalars (the window position, the context mask and size, the context
// mean), so that the caller's per-step state stays in registers.
struct HqlOut {
    float x[4];
    uint32_t mph;  // tensor-core barrier phase after the step
};

template <int MIXED>
__device__ __noinline__ HqlOut hql_step(const KParams& P, int wr, int wc,
                                        unsigned long long ymask, int ny, float mean, bool trace,
                                        uint32_t mph, float* ubuf) {
    Smem& sm = smem_ref();
    Hql& h = sm.hql;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int nz = ny + 4;
    const float shift = rintf(mean);
    StepCtx c;  // the parts of the step context the candidate test needs
    c.ymask = ymask;
#pragma unroll
    for (int r = 0; r < 6; ++r)
        c.rowcfg[r] = (unsigned)((ymask >> (6 * r)) & 63ull) | ((r == 2 || r == 3) ? 12u : 0u);

    // context lists (compacted, window raster order)
    if (tid < 36 && ((ymask >> tid) & 1ull)) {
        const int idx = __popcll(ymask & ((1ull << tid) - 1ull));
        h.off[idx] = (short)((tid / 6) * kReg + (tid % 6));
        h.ys[idx] = sm.S[(wr + tid / 6) * kReg + wc + tid % 6] - shift;
    }
    if (tid >= 64 && tid < 100 && tid - 64 >= ny) {  // zero padding of the lists
        h.off[tid - 64] = 0;
        h.ys[tid - 64] = 0.0f;
    }

    // H0: valid candidates, ascending window index (R5)
    {
        int cnt = 0;
        unsigned flags = 0;
        for (int q = 0; q < 8; ++q) {
            const int p = tid * 8 + q;
            if (p < kNcand) {
                const int u = p / kNpos, v = p - (p / kNpos) * kNpos;
                if (cand_valid(sm, c, u, v)) {
                    flags |= 1u << q;
                    ++cnt;
                }
            }
        }
        int total;
        int pos = block_exscan(cnt, h.scan, &total);  // (barriers: the lists above are visible)
        for (int q = 0; q < 8; ++q)
            if ((flags >> q) & 1u) {
                const int p = tid * 8 + q;
                h.cand[pos++] = (uint16_t)((p / kNpos) * kReg + (p % kNpos));
            }
        if (tid == 0) h.M = total;
        hql_build_koff(h, nz);
    }
    __syncthreads();
    const int M = h.M;
    const int nchunks = (M + kCh - 1) / kCh;
    SK_PHASE(PH_H0);

    // chunks (and MMA commits) of the tensor-core passes at the tuned tile sizes (the beta
    // pass keeps kCh)
    const int nch13 = (M + P.tile_h13 - 1) / P.tile_h13, nch2 = (M + P.tile_h2 - 1) / P.tile_h2;
    if (MIXED) {
        if (P.tile_h13 == 32) h1_mixed<MIXED == 1, 32>(M, nz, shift, sm.tmem_base, mph);
        else h1_mixed<MIXED == 1, 64>(M, nz, shift, sm.tmem_base, mph);
        mph ^= (uint32_t)(nch13 & 1);
    } else
    // H1: sums of z' and z' z'^T, z' = z - shift (Eq. (8)).  Thread (a, g) owns row a of the
    // product matrix over the candidates j = g (mod kG1).  Integer parts multiply and
    // accumulate exactly in int32 (|n| <= 255, at most 1849 products: < 2^31); fractional
    // cross terms accumulate in FP32 (they are small).
    {
        constexpr int kG1 = kThreads / 36;
        const int a = tid % 36, g = tid / 36;
        const bool act = g < kG1 && a < nz;
        int ai[36];
        float af[36];
#pragma unroll
        for (int b = 0; b < 36; ++b) {
            ai[b] = 0;
            af[b] = 0.0f;
        }
        int colN = 0;
        float colF = 0.0f;
        for (int idx = tid; idx < 36 * 36; idx += kThreads) {
            h.p1.cint[idx / 36][idx % 36] = 0;
            h.p1.cfrac[idx / 36][idx % 36] = 0.0f;
            if (idx < 36) h.colNi[idx] = 0;
        }
        const int* zi = reinterpret_cast<const int*>(&h.Z[0][0][0]);
        const float* zf = &h.Z[1][0][0];
        for (int ch = 0; ch < nchunks; ++ch) {
            const int c0 = ch * kCh, n = min(kCh, M - c0);
            if (ch > 0) __syncthreads();  // previous chunk consumed
            const bool frac = hql_stage_split(sm, c0, n, shift);
            const bool any_frac = __syncthreads_or(frac) != 0;
            if (act) {
                for (int j = g; j < n; j += kG1) {
                    const int na = zi[j * kZrow + a];
                    const float fa = zf[j * kZrow + a];
                    colN += na;
                    colF += fa;
#pragma unroll
                    for (int b4 = 0; b4 < 9; ++b4) {
                        const int4 nb = *reinterpret_cast<const int4*>(&zi[j * kZrow + 4 * b4]);
                        ai[4 * b4 + 0] += na * nb.x;
                        ai[4 * b4 + 1] += na * nb.y;
                        ai[4 * b4 + 2] += na * nb.z;
                        ai[4 * b4 + 3] += na * nb.w;
                    }
                    if (any_frac) {
                        const float naf = (float)na;
#pragma unroll
                        for (int b4 = 0; b4 < 9; ++b4) {
                            const int4 nb = *reinterpret_cast<const int4*>(&zi[j * kZrow + 4 * b4]);
                            const float4 fb = *reinterpret_cast<const float4*>(&zf[j * kZrow + 4 * b4]);
                            // n_a f_b + f_a (n_b + f_b)
                            af[4 * b4 + 0] = __fmaf_rn(naf, fb.x, __fmaf_rn(fa, (float)nb.x + fb.x, af[4 * b4 + 0]));
                            af[4 * b4 + 1] = __fmaf_rn(naf, fb.y, __fmaf_rn(fa, (float)nb.y + fb.y, af[4 * b4 + 1]));
                            af[4 * b4 + 2] = __fmaf_rn(naf, fb.z, __fmaf_rn(fa, (float)nb.z + fb.z, af[4 * b4 + 2]));
                            af[4 * b4 + 3] = __fmaf_rn(naf, fb.w, __fmaf_rn(fa, (float)nb.w + fb.w, af[4 * b4 + 3]));
                        }
                    }
                }
            }
        }
        __syncthreads();
        if (act) {
#pragma unroll
            for (int b = 0; b < 36; ++b)
                if (ai[b]) atomicAdd(&h.p1.cint[a][b], ai[b]);
            atomicAdd(&h.colNi[a], colN);
        }
        // fractional sums in a fixed order of the subsets (deterministic)
        for (int gg = 0; gg < kG1; ++gg) {
            if (act && g == gg) {
#pragma unroll
                for (int b = 0; b < 36; ++b) h.p1.cfrac[a][b] += af[b];
                h.colF[a] = (gg == 0) ? colF : h.colF[a] + colF;
            }
            __syncthreads();
        }
    }
    SK_PHASE(PH_H1);

    // finalise C_ab = S_ab/M - T_a T_b / M^2 in double-float; YY (+ridge later), XY
    {
        const df32 invM = df_div(df_make(1.0f), df_make((float)M));
        for (int idx = tid; idx < 36 * 36; idx += kThreads) {
            const int a = idx / 36, b = idx % 36;
            if (a > b || b < 4 || b >= nz) continue;
            const df32 S = df_add(df_from_int(h.p1.cint[a][b]), df_make(h.p1.cfrac[a][b]));
            const df32 Ta = df_add(df_from_int(h.colNi[a]), df_make(h.colF[a]));
            const df32 Tb = df_add(df_from_int(h.colNi[b]), df_make(h.colF[b]));
            const df32 Cab = df_sub(df_mul(S, invM), df_mul(df_mul(Ta, invM), df_mul(Tb, invM)));
            if (a >= 4) {
                h.p1.A[b - 4][a - 4] = Cab;  // lower triangle (row >= col)
            } else {
                h.cxy[a][b - 4] = Cab;
            }
        }
    }
    __syncthreads();
    // ridge (R7): lambda = ridge_rel * tr(C_YY)/Ny + 1e-6
    if (wid == 0) {
        df32 t = lane < ny ? h.p1.A[lane][lane] : df_make(0.0f);
        for (int o = 16; o > 0; o >>= 1) {
            df32 u;
            u.hi = __shfl_xor_sync(0xffffffffu, t.hi, o);
            u.lo = __shfl_xor_sync(0xffffffffu, t.lo, o);
            t = df_add(t, u);
        }
        const df32 lam = df_add(df_mul_f(df_div(t, df_make((float)ny)), P.ridge_rel), df_make(1e-6f));
        __syncwarp();
        if (lane < ny) h.p1.A[lane][lane] = df_add(h.p1.A[lane][lane], lam);
        if (lane == 0) h.lam = df_to_f(lam);
    }
    for (int idx = tid; idx < 32 * 33; idx += kThreads) h.p1.X[idx / 33][idx % 33] = df_make(0.0f);
    __syncthreads();

    // Cholesky / inverse factor in double-float: Gaussian elimination A = Lu D Lu^T and
    // the same row operations applied to I give X = Lu^-1; then L^-1 = D^-1/2 X.
    {
        constexpr int kPairs = 528;  // lower-triangle entries of a 32 x 32 matrix
        constexpr int kPer = (kPairs + kThreads - 1) / kThreads;
        int pi[kPer], pj[kPer];
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const int p = tid + q * kThreads;
            int i = (int)((sqrtf(8.0f * p + 1.0f) - 1.0f) * 0.5f);
            while ((i + 1) * (i + 2) / 2 <= p) ++i;
            while (i * (i + 1) / 2 > p) --i;
            pi[q] = (p < kPairs) ? i : 99;
            pj[q] = p - i * (i + 1) / 2;
        }
        for (int k = 0; k < ny; ++k) {
            const df32 akk = h.p1.A[k][k];
            const df32 rinv = df_rcp(akk);
#pragma unroll
            for (int q = 0; q < kPer; ++q) {
                const int i = pi[q], j = pj[q];
                if (i >= ny || i <= k) continue;
                const df32 mlt = df_mul(h.p1.A[i][k], rinv);
                if (j > k) {
                    h.p1.A[i][j] = df_sub(h.p1.A[i][j], df_mul(mlt, h.p1.A[j][k]));
                } else if (j == k) {
                    h.p1.X[i][k] = df_neg(mlt);
                } else {
                    h.p1.X[i][j] = df_sub(h.p1.X[i][j], df_mul(mlt, h.p1.X[k][j]));
                }
            }
            __syncthreads();
        }
        // L^-1 = D^-1/2 X: kept in double-float in X, rounded to FP32 in Linv.  The row scales
        // D^-1/2 once per row (in ebard, free until the beta pass).
        if (tid < 32) h.ebard[tid] = tid < ny ? df_rcp(df_sqrt(h.p1.A[tid][tid])) : df_make(0.0f);
        __syncthreads();
        for (int idx = tid; idx < 32 * 32; idx += kThreads) {
            const int i = idx >> 5, j = idx & 31;
            float v = 0.0f;
            if (i < ny && j <= i) {
                const df32 rs = h.ebard[i];
                const df32 l = (j == i) ? rs : df_mul(h.p1.X[i][j], rs);
                v = df_to_f(l);
                h.p1.X[i][j] = l;
            }
            h.Linv[i][j] = v;
        }
    }
    __syncthreads();
    // G = C_XY L^-T (4 x ny): G[a][i] = sum_k C_XY[a][k] Linv[i][k], in double-float;
    // kept in FP32 for the leave-one-out corrections and in double-float (in the first
    // rows of A, no longer needed) for K.  Thread (a, i, half): the sums over k < 16 and
    // k >= 16 in adjacent lanes, added as (lower half) + (upper half) in both.
    {
        const int half = tid & 1, i = (tid >> 1) & 31, a = tid >> 6;
        df32 g = df_make(0.0f);
        if (i < ny) {
            const int k1 = min(i, half ? 31 : 15);
            for (int k = half ? 16 : 0; k <= k1; ++k) g = df_add(g, df_mul(h.cxy[a][k], h.p1.X[i][k]));
        }
        df32 o;
        o.hi = __shfl_xor_sync(0xffffffffu, g.hi, 1);
        o.lo = __shfl_xor_sync(0xffffffffu, g.lo, 1);
        g = half ? df_add(o, g) : df_add(g, o);
        __syncthreads();  // every read of A (and of X) for G done before A's rows take G
        if (half == 0) {
            h.G[a][i] = df_to_f(g);
            h.p1.A[a][i] = g;
        }
    }
    __syncthreads();
    // K = C_XY C_YY^-1 = G L^-1: K[a][j] = sum_{i >= j} G[a][i] Linv[i][j] (double-float),
    // split over i < 16 and i >= 16 in the same way
    {
        const int half = tid & 1, j = (tid >> 1) & 31, a = tid >> 6;
        df32 kk = df_make(0.0f);
        if (j < ny) {
            const int i1 = half ? ny - 1 : min(15, ny - 1);
            for (int i = max(j, half ? 16 : 0); i <= i1; ++i) kk = df_add(kk, df_mul(h.p1.A[a][i], h.p1.X[i][j]));
        }
        df32 o;
        o.hi = __shfl_xor_sync(0xffffffffu, kk.hi, 1);
        o.lo = __shfl_xor_sync(0xffffffffu, kk.lo, 1);
        kk = half ? df_add(o, kk) : df_add(kk, o);
        if (half == 0) {
            h.K[a][j] = kk;
            h.Kf[a][j] = df_to_f(kk);
        }
    }
    SK_PHASE(PH_CHOL);

    // H2: whitened distances d_j = ||L^-1 (y_j - y0)||^2 (Mahalanobis, Eq. (6) with C_YY)
    // thread tile: 2 candidates x 4 whitened coordinates
    const int tj = (tid >> 3) * 2, tq = tid & 7;
    float lmin = INFINITY;
    if (MIXED) {
        if (P.tile_h2 == 128) lmin = h2_mixed<MIXED == 1, 128>(M, ny, shift, sm.tmem_base, mph, ubuf);
        else lmin = h2_mixed<MIXED == 1, 64>(M, ny, shift, sm.tmem_base, mph, ubuf);
        mph ^= (uint32_t)(nch2 & 1);
    } else {
        hql_stage(sm, 0, 0, min(kCh, M), shift);
        for (int ch = 0; ch < nchunks; ++ch) {
            const int buf = ch & 1, c0 = ch * kCh, n = min(kCh, M - c0);
            __syncthreads();
            float u0[4], u1[4];
            whiten_tile(h, buf, ny, tj, tq, u0, u1);
            if (4 * tq >= ny) {  // coordinates past Ny: zero, not stored
            } else if (tj < n)
                *reinterpret_cast<float4*>(ubuf + (size_t)(c0 + tj) * kMaxNy + ubuf_pos(c0 + tj, tq)) =
                    make_float4(u0[0], u0[1], u0[2], u0[3]);
            if (4 * tq < ny && tj + 1 < n)
                *reinterpret_cast<float4*>(ubuf + (size_t)(c0 + tj + 1) * kMaxNy + ubuf_pos(c0 + tj + 1, tq)) =
                    make_float4(u1[0], u1[1], u1[2], u1[3]);
            float p0 = 0.0f, p1 = 0.0f;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                p0 = __fmaf_rn(u0[q], u0[q], p0);
                p1 = __fmaf_rn(u1[q], u1[q], p1);
            }
#pragma unroll
            for (int o = 4; o > 0; o >>= 1) {
                p0 += __shfl_xor_sync(0xffffffffu, p0, o);
                p1 += __shfl_xor_sync(0xffffffffu, p1, o);
            }
            if (tq == 0) {
                if (tj < n) {
                    h.d[c0 + tj] = p0;
                    lmin = fminf(lmin, p0);
                }
                if (tj + 1 < n) {
                    h.d[c0 + tj + 1] = p1;
                    lmin = fminf(lmin, p1);
                }
            }
            if (ch + 1 < nchunks) hql_stage(sm, buf ^ 1, c0 + kCh, min(kCh, M - c0 - kCh), shift);
        }
    }
    lmin = warp_max(-lmin);
    if (lane == 0) h.red[wid][0] = -lmin;
    __syncthreads();
    if (tid == 0) {
        float mn = h.red[0][0];
        for (int w = 1; w < kWarps; ++w) mn = fminf(mn, h.red[w][0]);
        h.dmin = mn;
    }
    __syncthreads();
    const float dmin = h.dmin;
    SK_PHASE(PH_H2);

    // H3: beta grid, Eqs. (9)-(10).  Thread (b, g) owns beta_b over the candidates
    // j = g (mod kG3): acc[k] = sum_j w_j(b) z'_j[k] for the staged columns (x', y', 1).
    // Subset partial sums merge in double-float.
    const int nb = P.nbeta;
    if (MIXED) {
        h3_mixed<MIXED == 1>(P, M, nz, shift, dmin, sm.tmem_base, mph);
        mph ^= (uint32_t)(nchunks & 1);
    } else {
        const int G3 = kThreads / nb;
        const int kql3 = (nz + 3) / 4;  // live column quads: 0 .. nz-1, and the constant (9)
        const int b = tid % nb, g = tid / nb;
        const bool act = g < G3;
        const float ib = P.inv2beta[b];
        float acc[kZs];
#pragma unroll
        for (int k = 0; k < kZs; ++k) acc[k] = 0.0f;
        hql_stage(sm, 0, 0, min(kCh, M), shift);
        for (int ch = 0; ch < nchunks; ++ch) {
            const int buf = ch & 1, c0 = ch * kCh, n = min(kCh, M - c0);
            __syncthreads();
            if (act) {
                for (int j = g; j < n; j += G3) {
                    const float w = __expf(-(h.d[c0 + j] - dmin) * ib);
#pragma unroll
                    for (int k4 = 0; k4 < kZs / 4; ++k4) {
                        if (k4 >= kql3 && k4 != 9) continue;  // columns past the context are zero
                        const float4 z = *reinterpret_cast<const float4*>(&h.Z[buf][j][4 * k4]);
                        acc[4 * k4 + 0] = __fmaf_rn(w, z.x, acc[4 * k4 + 0]);
                        acc[4 * k4 + 1] = __fmaf_rn(w, z.y, acc[4 * k4 + 1]);
                        acc[4 * k4 + 2] = __fmaf_rn(w, z.z, acc[4 * k4 + 2]);
                        acc[4 * k4 + 3] = __fmaf_rn(w, z.w, acc[4 * k4 + 3]);
                    }
                }
            }
            if (ch + 1 < nchunks) hql_stage(sm, buf ^ 1, c0 + kCh, min(kCh, M - c0 - kCh), shift);
        }
        __syncthreads();
        if (act) {
#pragma unroll
            for (int k = 0; k < 37; ++k) h.p2.mrg[tid][k] = acc[k];
        }
        __syncthreads();
        for (int idx = tid; idx < nb * 37; idx += kThreads) {
            const int bb = idx / 37, k = idx % 37;
            df32 s = df_make(0.0f);
            for (int gg = 0; gg < G3; ++gg) s = df_add(s, df_make(h.p2.mrg[gg * nb + bb][k]));
            h.accBd[bb][k] = s;
        }
    }
    __syncthreads();
    // eps_y(b) = || y0 - y~0(b) ||^2 ; warp w handles b = w, w+8, ...
    for (int b = wid; b < nb; b += kWarps) {
        float e = 0.0f;
        if (lane < ny) {
            const df32 r = df_sub(df_div(h.accBd[b][4 + lane], h.accBd[b][36]), df_make(h.ys[lane]));
            const float rf = df_to_f(r);
            e = rf * rf;
        }
        e = warp_sum(e);
        if (lane == 0) h.eps[b] = e;
    }
    __syncthreads();
    if (tid == 0) {
        float emin = h.eps[0];
        for (int b = 1; b < nb; ++b) emin = fminf(emin, h.eps[b]);
        int bs = 0;
        for (int b = 0; b < nb; ++b)
            if (h.eps[b] <= emin * (1.0f + P.beta_tie_rel)) {
                bs = b;
                break;
            }
        h.bstar = bs;
    }
    __syncthreads();
    const int bstar = h.bstar;
    // x~0 and e-bar = y~0 - y0 (relative to the shift) at beta*, Eqs. (4)-(5)
    if (tid < 36) {
        const df32 sw = h.accBd[bstar][36];
        if (tid < 4) h.xt0d[tid] = df_div(h.accBd[bstar][tid], sw);
        else if (tid - 4 < ny) h.ebard[tid - 4] = df_sub(df_div(h.accBd[bstar][tid], sw), df_make(h.ys[tid - 4]));
    }
    __syncthreads();
    // the correction of Eq. (13): K (y0 - y~0) = -K e-bar (double-float)
    if (wid == 0) {
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            df32 t = (lane < ny) ? df_mul(h.K[a][lane], h.ebard[lane]) : df_make(0.0f);
            for (int o = 16; o > 0; o >>= 1) {
                df32 u;
                u.hi = __shfl_xor_sync(0xffffffffu, t.hi, o);
                u.lo = __shfl_xor_sync(0xffffffffu, t.lo, o);
                t = df_add(t, u);
            }
            if (lane == 0) h.corr[a] = df_neg(t);
        }
    }
    SK_PHASE(PH_H3);

    // H4: I0 = the n0 smallest d_j, ties to the lower index (radix select on the bits)
    int n0 = min(ny + 1, M - 1);
    if (n0 < 0) n0 = 0;
    if (n0 > 0) {
        unsigned prefix = 0, maskbits = 0;
        int need = n0;
        for (int i = tid; i < 256; i += kThreads) h.hist[0][i] = 0;
        __syncthreads();
        for (int shiftb = 24, pb = 0; shiftb >= 0; shiftb -= 8, pb ^= 1) {
            for (int j = tid; j < M; j += kThreads) {
                const unsigned key = __float_as_uint(h.d[j]);
                if ((key & maskbits) == prefix) atomicAdd(&h.hist[pb][(key >> shiftb) & 255u], 1);
            }
            __syncthreads();
            if (wid == 0) {
                // first digit whose cumulative count reaches `need` (warp scan of 8 bins/lane)
                int loc[8], s8 = 0;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    loc[q] = h.hist[pb][lane * 8 + q];
                    s8 += loc[q];
                }
                int incl = s8;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                const int excl = incl - s8;
                const unsigned hit = __ballot_sync(0xffffffffu, incl >= need);
                const int src = __ffs(hit) - 1;
                if (lane == src) {
                    int acc = excl, dg = lane * 8;
                    for (int q = 0; q < 8; ++q) {
                        if (acc + loc[q] >= need) {
                            dg = lane * 8 + q;
                            break;
                        }
                        acc += loc[q];
                    }
                    h.sel[pb][0] = dg;
                    h.sel[pb][1] = need - acc;
                }
            } else {  // the next pass's histogram (its last reader was two barriers ago)
                for (int i = tid - 32; i < 256; i += kThreads - 32) h.hist[pb ^ 1][i] = 0;
            }
            __syncthreads();
            prefix |= (unsigned)h.sel[pb][0] << shiftb;
            maskbits |= 255u << shiftb;
            need = h.sel[pb][1];
        }
        // members: key < prefix, plus the first `need` with key == prefix (index order)
        unsigned f = 0, eqf = 0;
        const int per = (M + kThreads - 1) / kThreads;  // <= 8
        for (int q = 0; q < per; ++q) {
            const int j = tid * per + q;
            if (j < M) {
                const unsigned key = __float_as_uint(h.d[j]);
                if (key < prefix) f |= 1u << q;
                if (key == prefix) eqf |= 1u << q;
            }
        }
        int tot;
        int eqpos = block_exscan(__popc(eqf), h.scan, &tot);
        unsigned take = f;
        for (int q = 0; q < per; ++q)
            if ((eqf >> q) & 1u) {
                if (eqpos < need) take |= 1u << q;
                ++eqpos;
            }
        int pos = block_exscan(__popc(take), h.scan, &tot);
        for (int q = 0; q < per; ++q)
            if ((take >> q) & 1u) h.i0[pos++] = tid * per + q;
        __syncthreads();
        // UI = L^-1 (y_i - y0) of the members, as the distance pass formed them; XI = x_i - shift
        for (int idx = tid; idx < kMaxI0 * 36; idx += kThreads) {
            const int i = idx / 36, k = idx % 36;
            if (i >= n0) continue;
            if (k < 32) {
                const int jj = h.i0[i];
                h.UI[i][k] = k < ny ? __ldcg(ubuf + (size_t)jj * kMaxNy + ubuf_pos(jj, k >> 2) + (k & 3)) : 0.0f;
            } else {
                const int base = h.cand[h.i0[i]];
                const int a = k - 32;
                h.XI[i][a] = sm.S[base + (a >> 1) * kReg + (a & 1) + 2 * kReg + 2] - shift;
            }
        }
    }
    __syncthreads();
    SK_PHASE(PH_H4);

    // H5: leave-one-out predictions for i in I0 at beta* (Eqs. (11)-(12)): for each member i
    // the online max-subtracted softmax of -||u_i - u_j||^2 / (2 beta*) over the candidates
    // j != i, and the weighted sums of [x'_j | G u_j | 1].  The correction G (u_i - u~_i) of
    // Eq. (11) is linear in u, and G u_j = G L^-1 (y_j - y0) = K (y_j - y0), so four columns
    // of G u_j stand in for the 32 of u_j in the sums.  Each warp owns every 8th group of 32
    // candidates and runs without CTA barriers until the merge:
    //   candidate mode (lane = candidate j): u_j = L^-1 (y_j - y0) as the distance pass
    //     formed it (read back from ubuf), K (y_j - y0) = G u_j and x'_j into the warp's
    //     buffer;
    //   member mode (lane = member i < 32): the buffered candidates in turn, the squared
    //     whitened distance in packed two-lane FP32 over coordinate pairs;
    //   member 32 (|I0| = 33): each lane keeps the sums of its own candidates.
    float num = 0.0f, den = 0.0f;
    if (n0 > 0) {
        const float ib = P.inv2beta[bstar];
        const int nbat = (M + 31) >> 5;
        // whitened coordinates in groups of 4: past Ny they are exact zeros (L^-1 and the
        // members' u_i are zero there), so member mode sums only the first nq groups, with
        // the results of all 8 bit for bit
        const int nq = (ny + 3) >> 2;
        float(*wb)[kWb] = h.h5.Wb[wid];
        const bool has32 = n0 > 32;
        const int selfi = lane < n0 ? h.i0[lane] : -1;
        const int self32 = has32 ? h.i0[32] : -1;
        float m = -INFINITY, sw = 0.0f, sa[8];  // member mode: member `lane`
        float m3 = -INFINITY, s3 = 0.0f, a3[8];  // member 32 over this lane's candidates
#pragma unroll
        for (int k = 0; k < 8; ++k) sa[k] = a3[k] = 0.0f;
        for (int bt = wid; bt < nbat; bt += kWarps) {
            const int j = 32 * bt + lane;
            const bool live = j < M;
            {   // candidate mode: the group's u_j (from the distance pass) into the buffer,
                // then per lane K (y_j - y0) = G u_j and x'_j
                const float* src = ubuf + (size_t)32 * bt * kMaxNy;
                const int nrow = min(32, M - 32 * bt);
#pragma unroll
                for (int t = 0; t < 8; ++t) {  // 4 KB, coalesced; a quarter-warp fills one row
                    const int idx = lane + 32 * t, row = idx >> 3, c4 = idx & 7;
                    const float4 v = (row < nrow && c4 < nq)
                                         ? __ldcg(reinterpret_cast<const float4*>(src + row * kMaxNy + ubuf_pos(row, c4)))
                                         : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                    *reinterpret_cast<float4*>(&wb[row][12 + 4 * c4]) = v;
                }
                __syncwarp();
                const int base = live ? h.cand[j] : 0;
                float g[4] = {0.0f, 0.0f, 0.0f, 0.0f};  // G u_j over the live coordinate groups
                for (int q = 0; q < nq; ++q) {
                    const float4 uv = *reinterpret_cast<const float4*>(&wb[lane][12 + 4 * q]);
#pragma unroll
                    for (int aa = 0; aa < 4; ++aa) {
                        const float4 gv = *reinterpret_cast<const float4*>(&h.G[aa][4 * q]);
                        g[aa] = __fmaf_rn(gv.x, uv.x, g[aa]);
                        g[aa] = __fmaf_rn(gv.y, uv.y, g[aa]);
                        g[aa] = __fmaf_rn(gv.z, uv.z, g[aa]);
                        g[aa] = __fmaf_rn(gv.w, uv.w, g[aa]);
                    }
                }
                float x[4];
#pragma unroll
                for (int aa = 0; aa < 4; ++aa)
                    x[aa] = live ? sm.S[base + (aa >> 1) * kReg + (aa & 1) + 2 * kReg + 2] - shift : 0.0f;
                *reinterpret_cast<float4*>(&wb[lane][0]) = make_float4(x[0], x[1], x[2], x[3]);
                *reinterpret_cast<float4*>(&wb[lane][4]) = make_float4(g[0], g[1], g[2], g[3]);
                if (has32 && live && j != self32) {  // member 32 against this candidate
                    f32x2 d2 = 0ull;
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(&wb[lane][12 + 4 * q]);
                        const ulonglong2 w = *reinterpret_cast<const ulonglong2*>(&h.UI[32][4 * q]);
                        f32x2 t = f2_sub(w.x, v.x);
                        d2 = f2_fma(t, t, d2);
                        t = f2_sub(w.y, v.y);
                        d2 = f2_fma(t, t, d2);
                    }
                    float dl, dh;
                    f2_unpack(d2, dl, dh);
                    h5_online(-(dl + dh) * ib, make_float4(x[0], x[1], x[2], x[3]),
                              make_float4(g[0], g[1], g[2], g[3]), m3, s3, a3);
                }
            }
            __syncwarp();
            if (lane < n0) {  // member mode, unrolled over the live coordinate groups
                const int nc = min(32, M - 32 * bt);
                if (nq <= 4) h5_members<4>(wb, h.UI[lane], nc, selfi - 32 * bt, ib, m, sw, sa);
                else if (nq <= 5) h5_members<5>(wb, h.UI[lane], nc, selfi - 32 * bt, ib, m, sw, sa);
                else h5_members<8>(wb, h.UI[lane], nc, selfi - 32 * bt, ib, m, sw, sa);
            }
            __syncwarp();  // the buffer takes the next group
        }
        // the warps' partial sums: member mode, and member 32 reduced over the lanes
        if (lane < n0) {
            float* mg = h.h5.Mg[wid][lane];
            mg[0] = m;
            mg[1] = sw;
#pragma unroll
            for (int k = 0; k < 8; ++k) mg[2 + k] = sa[k];
        }
        if (has32) {
            float wm = m3;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) wm = fmaxf(wm, __shfl_xor_sync(0xffffffffu, wm, o));
            const float sc = m3 == -INFINITY ? 0.0f : __expf(m3 - wm);
            float v9[9];
            v9[0] = s3 * sc;
#pragma unroll
            for (int k = 0; k < 8; ++k) v9[1 + k] = a3[k] * sc;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                for (int k = 0; k < 9; ++k) v9[k] += __shfl_xor_sync(0xffffffffu, v9[k], o);
            if (lane == 0) {
                float* mg = h.h5.Mg[wid][32];
                mg[0] = wm;
#pragma unroll
                for (int k = 0; k < 9; ++k) mg[1 + k] = v9[k];
            }
        }
        __syncthreads();
        // merge over the warps: accI[i] = x' sums (0..3), G u sums (4..7), weight sum (8)
        for (int idx = tid; idx < n0 * 9; idx += kThreads) {
            const int i = idx / 9, k = idx - (idx / 9) * 9;
            float mx = -INFINITY;
#pragma unroll
            for (int w = 0; w < kWarps; ++w) mx = fmaxf(mx, h.h5.Mg[w][i][0]);
            const int col = k == 8 ? 1 : 2 + k;
            float acc = 0.0f;
#pragma unroll
            for (int w = 0; w < kWarps; ++w) {
                const float mw = h.h5.Mg[w][i][0];
                if (mw != -INFINITY) acc = __fmaf_rn(__expf(mw - mx), h.h5.Mg[w][i][col], acc);
            }
            h.accI[i][k] = acc;
        }
        __syncthreads();
        // r_i = x_i - x~_i ; g_i = G u_i - (sum_j w_ij G u_j) / sum_j w_ij ;
        // alpha = sum r.g / sum g.g
        if (tid < 4 * kMaxI0) {
            const int i = tid >> 2, aa = tid & 3;
            if (i < n0) {
                const float inv = 1.0f / h.accI[i][8];
                const float r = h.XI[i][aa] - h.accI[i][aa] * inv;
                float gu = 0.0f;
                for (int k = 0; k < ny; ++k) gu = __fmaf_rn(h.G[aa][k], h.UI[i][k], gu);
                const float gg = gu - h.accI[i][4 + aa] * inv;
                num = r * gg;
                den = gg * gg;
            }
        }
    }
    SK_PHASE(PH_H5);
    num = warp_sum(num);
    den = warp_sum(den);
    __syncthreads();
    if (lane == 0) {
        h.red[wid][0] = num;
        h.red[wid][1] = den;
    }
    __syncthreads();
    if (tid == 0) {
        float nn = 0.0f, dd = 0.0f;
        for (int w = 0; w < kWarps; ++w) {
            nn += h.red[w][0];
            dd += h.red[w][1];
        }
        float al = dd > 0.0f ? nn / dd : 0.0f;
        al = fminf(fmaxf(al, 0.0f), 1.0f);
        h.alpha = al;
        h.n0 = n0;
    }
    __syncthreads();
    const float alpha = h.alpha;
    // x0_hat = x~0 + alpha C_XY C_YY^-1 (y0 - y~0), Eq. (13)
    HqlOut out;
    out.mph = mph;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const df32 v = df_add(df_add(df_make(shift), h.xt0d[a]), df_mul_f(h.corr[a], alpha));
        out.x[a] = df_to_f(v);
    }
    if (trace && tid == 0) {
        sm.tr.beta_idx = (int8_t)bstar;
        sm.tr.n0 = (int8_t)n0;
        sm.tr.alpha = alpha;
        sm.tr.eps_best = h.eps[bstar];
        sm.tr.m = (int16_t)M;
        for (int t = 0; t < 36; ++t) {
            if (t < n0) {
                const int base = h.cand[h.i0[t]];
                sm.tr.i0[t] = (uint16_t)((base / kReg) * kNpos + base % kReg);
            } else {
                sm.tr.i0[t] = 0xffff;
            }
        }
    }
    if (tid == 0) {
        sm.st[ST_HQL_M] += M;
        sm.st[ST_HQL_MNY] += (unsigned long long)M * ny;
        sm.st[ST_HQL_I0M] += (unsigned long long)n0 * M;
        sm.st[ST_HQL_MNY2] += (unsigned long long)M * ny * ny;
        sm.st[ST_HQL_NY3] += (unsigned long long)ny * ny * ny;
        sm.st[ST_HQL_I0MNY] += (unsigned long long)n0 * M * ny;
#ifdef SKMMSE_PHASE_CLOCKS
        {
            const long long t_ = clock64();
            sm.st[kPhaseBase + PH_HFIN] += (unsigned long long)(t_ - sm.ph_t);
            sm.ph_t = t_;
        }
#endif
        // algorithmic FP32 operations of this HQL estimate (one exp counts as one):
        // covariance (upper C_YY and C_XY), whitening with the distance, beta grid (exp +
        // weighted sums of 4+Ny+1 columns), leave-one-out pass
        const unsigned long long Mu = M, nyu = ny, n0u = n0, nbu = P.nbeta;
        sm.st[ST_FLOPS] += Mu * (nyu * (nyu + 1) + 8 * nyu + 2 * (nyu + 4)) +
                           Mu * (nyu * (nyu + 1) + 2 * nyu) +
                           nbu * Mu * (2 * (nyu + 5) + 3) +
                           n0u * Mu * (3 * nyu + 2 * (nyu + 5) + 3);
    }
    __syncthreads();
    return out;
}

// ------------------------------------------------------------------------------------
// the persistent kernel

// ------------------------------------------------------------------------------------
// Ready queue (see the work-queue notes below the kernel).  Called by warp 0 of a CTA;
// returns the claimed entry, -1 when every entry is claimed, -2 on a timeout (error word
// set).  The bound counts idle rounds without progress of the whole call.
__device__ __noinline__ int claim_ready(const WorkDev& W, int n_entries, unsigned idle_limit) {
    const int lane = threadIdx.x & 31;
    unsigned idle = 0;
    int seen = -1;
    for (;;) {
        const int claimed = ld_relaxed_i(&W.counters[1]);
        const int k0 = ld_relaxed_i(&W.counters[3]);  // (issued before the test: one round trip)
        if (claimed >= n_entries) return -1;
        if (claimed != seen) {
            seen = claimed;
            idle = 0;
        }
        bool lost_race = false;
        for (int kb = k0; kb < W.nbk; kb += 32) {
            const int k = kb + lane;
            int hd = 0, tl = 0, cnt = 0;
            if (k < W.nbk) {
                hd = ld_relaxed_i(&W.bk_head[k]);
                tl = ld_relaxed_i(&W.bk_tail[k]);
                cnt = W.bk_cnt[k];
            }
            const unsigned ready = __ballot_sync(0xffffffffu, k < W.nbk && hd < tl);
            if (kb == k0) {  // buckets fully claimed at the front never refill: move the start
                const unsigned drained = __ballot_sync(0xffffffffu, k >= W.nbk || hd >= cnt);
                const int adv = drained == 0xffffffffu ? 32 : __ffs(~drained) - 1;
                if (adv > 0 && lane == 0) atomicMax(&W.counters[3], kb + adv);
            }
            if (ready) {
                const int src = __ffs(ready) - 1;
                int pos = -1;
                if (lane == src) {
                    // a lost race returns the head another claimer left: while it is still
                    // below the tail seen (the tail only grows), try again on the same bucket
                    int h = hd;
                    for (int t = 0; t < 64 && h < tl; ++t) {
                        const int old = atomicCAS(&W.bk_head[k], h, h + 1);
                        if (old == h) {
                            pos = W.bk_off[k] + h;
                            break;
                        }
                        h = old;
                    }
                }
                pos = __shfl_sync(0xffffffffu, pos, src);
                if (pos < 0) {
                    lost_race = true;
                    break;
                }
                int e = -1;
                if (lane == 0) {
                    atomicAdd(&W.counters[1], 1);
                    // the publisher advances the tail just before it writes the slot
                    unsigned it = 0;
                    while ((e = ld_acquire_i(&W.slots[pos])) < 0) {
                        __nanosleep(32);
                        if (++it > (1u << 24)) {
                            atomicExch(&W.counters[2], 6);
                            break;
                        }
                    }
                }
                e = __shfl_sync(0xffffffffu, e, 0);
                return e < 0 ? -2 : e;
            }
        }
        if (lost_race) continue;
        __nanosleep(256);
        if (++idle > idle_limit) {
            if (lane == 0) atomicExch(&W.counters[2], 6);
            return -2;
        }
    }
}

// entry e (block mb of frame F) is done: count it off at each dependant and publish the
// dependants that became ready.  One thread.
__device__ __noinline__ void release_dependants(const WorkDev& W, const FrameDev& F, int mb) {
    const int y = mb / F.mbw, x = mb - (mb / F.mbw) * F.mbw;
    __threadfence();  // the done flag before the counts
    const int dys[4] = {0, 1, 1, 1}, dxs[4] = {1, -1, 0, 1};
    for (int t = 0; t < 4; ++t) {
        const int yy = y + dys[t], xx = x + dxs[t];
        if (yy >= F.mbh || xx < 0 || xx >= F.mbw) continue;
        const int qe = W.entry_of_mb[F.mb_base + yy * F.mbw + xx];
        if (qe < 0) continue;
        if (atomicSub(&W.rem[qe], 1) == 1) {
            __threadfence();
            const int key = W.entries[qe].w;
            const int k = atomicAdd(&W.bk_tail[key], 1);
            st_release_i(&W.slots[W.bk_off[key] + k], qe);
        }
    }
}

// tensor-memory columns per CTA: H1 uses 0..47, 64..111 and 128..175 (two CTAs per SM
// take the SM's 512 columns)
template <int MIXED>
constexpr uint32_t kTmemCols = 256u;

template <int MIXED, bool IDLTC = false>
__global__ void __launch_bounds__(kThreads, 2) conceal_kernel(const __grid_constant__ WorkDev W,
                                                              const __grid_constant__ KParams P) {
    Smem& sm = smem_ref();
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const bool trace_on = (P.flags & 1u) != 0u;
    const bool force_on = (P.flags & 2u) != 0u;
    const bool quant_on = (P.flags & 4u) != 0u;  // in-loop 8-bit quantisation

    if (tid == 0) {
        mbar_init(&sm.mbar, 1);
        tc::mbar_init(&sm.mma_bar, 1);
        sm.mma_err = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int i = tid; i < kNStats; i += kThreads) sm.st[i] = 0;
    if (MIXED && wid == 0) tc::tmem_alloc(&sm.tmem_base, kTmemCols<MIXED>);  // 128 lanes x FP32 columns
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    uint32_t mph = 0;
    unsigned phase = 0;
    const int n_entries = W.counters[0];
    if (tid == 0) {
        sm.ph_t = clock64();
        sm.st[ST_T_FIRST_INV] = ~globaltimer_ns();  // (slots cleared before the barrier above)
    }

    for (;;) {
        if (wid == 0) {
            const int got = claim_ready(W, n_entries, P.claim_idle_limit);
            if (lane == 0) sm.entry = got;
        }
        __syncthreads();
        const int e = sm.entry;
        if (e < 0) break;
        const int4 ent = W.entries[e];
        const FrameDev& F = W.frames[ent.x];
        const int mb = ent.y, mby = mb / F.mbw, mbx = mb - (mb / F.mbw) * F.mbw;
        const int oy = mby * kMB - kMB, ox = mbx * kMB - kMB;

        // neighbour status (R1)
        if (tid < 9) {
            const int ny_ = mby + tid / 3 - 1, nx_ = mbx + tid % 3 - 1;
            int st = 2, en = -1;
            if (ny_ >= 0 && nx_ >= 0 && ny_ < F.mbh && nx_ < F.mbw) {
                const int q = F.mb_base + ny_ * F.mbw + nx_;
                const int qe = W.entry_of_mb[q];
                if (qe < 0) st = 0;
                else if (P.concealed_is_support && (ny_ * F.mbw + nx_) < mb) {
                    st = 1;
                    en = qe;
                }
            }
            sm.nbst[tid] = st;
            sm.nbent[tid] = en;
        }
        // TMA: the 48x48 region of the 8-bit frame (out-of-frame reads fill zeros)
        if (tid == 0 && F.use_tma) {
            tmap_acquire(&W.tmaps[ent.x]);
            mbar_expect_tx(&sm.mbar, kReg * kReg);
            tma_load_2d(sm.raw, &W.tmaps[ent.x], &sm.mbar, ox, oy);
        }
        __syncthreads();
        // dependency waits (bounded)
        if (tid < 9 && sm.nbst[tid] == 1) {
            const unsigned* flag = &W.done[sm.nbent[tid]];
            unsigned it = 0;
            while (ld_acquire(flag) == 0u) {
                __nanosleep(200);
                if (++it > (1u << 25)) {
                    atomicExch(&W.counters[2], 6);
                    sm.nbst[tid] = 2;
                    break;
                }
            }
        }
        if (tid == 0 && F.use_tma) {
            if (!mbar_wait(&sm.mbar, phase, 1u << 26)) {
                atomicExch(&W.counters[2], 6);
                mbar_wait(&sm.mbar, phase, 1u << 26);
            }
        }
        phase ^= (F.use_tma ? 1u : 0u);
        __syncthreads();
        // convert to values + availability (ballot per row half).  A warp takes rows wid,
        // wid + 8, ..., every value of its 6 rows read (the dependencies' values from L2)
        // before any is stored.
        {
            constexpr int kRows = kReg / kWarps;
            float v[kRows][2];
            bool av[kRows][2];
#pragma unroll
            for (int q = 0; q < kRows; ++q) {
                const int r = wid + kWarps * q;
#pragma unroll
                for (int half = 0; half < 2; ++half) {
                    const int cc = half * 32 + lane;
                    bool a = false;
                    float x = 0.0f;
                    if (cc < kReg) {
                        const int fy = oy + r, fx = ox + cc;
                        if (fy >= 0 && fx >= 0 && fy < F.h && fx < F.w) {
                            const int nb = (r / kMB) * 3 + cc / kMB;
                            const int st = sm.nbst[nb];
                            if (st == 0) {
                                x = F.use_tma ? (float)sm.raw[r * kReg + cc]
                                              : (float)F.in[(size_t)fy * F.pitch + fx];
                                a = true;
                            } else if (st == 1) {
                                x = __ldcg(&W.vals[(size_t)sm.nbent[nb] * 256 + (r % kMB) * kMB + cc % kMB]);
                                a = true;
                            } else if (F.px_lost && F.px_lost[(size_t)fy * F.px_pitch + fx] == 0) {
                                // a received pixel of a lost block (per-pixel loss)
                                x = F.use_tma ? (float)sm.raw[r * kReg + cc]
                                              : (float)F.in[(size_t)fy * F.pitch + fx];
                                a = true;
                            }
                        }
                    }
                    v[q][half] = x;
                    av[q][half] = a;
                }
            }
#pragma unroll
            for (int q = 0; q < kRows; ++q) {
                const int r = wid + kWarps * q;
                unsigned long long bits = 0;
#pragma unroll
                for (int half = 0; half < 2; ++half) {
                    const int cc = half * 32 + lane;
                    if (cc < kReg) sm.S[r * kReg + cc] = v[q][half];
                    bits |= (unsigned long long)__ballot_sync(0xffffffffu, av[q][half]) << (32 * half);
                }
                if (lane == 0) sm.av[r] = bits;
            }
        }
        __syncthreads();
        if (wid == 0) {  // patches to fill: in the frame, holding a lost (unavailable) pixel
            unsigned bal[2];
#pragma unroll
            for (int h2 = 0; h2 < 2; ++h2) {  // lane l: patches l and l + 32
                const int p = lane + 32 * h2, a = p >> 3, b = p & 7;
                const int pr = kMB + 2 * a, pc = kMB + 2 * b;
                const bool full = ((sm.av[pr] >> pc) & 3ull) == 3ull && ((sm.av[pr + 1] >> pc) & 3ull) == 3ull;
                bal[h2] = __ballot_sync(0xffffffffu, mby * kMB + 2 * a < F.h && mbx * kMB + 2 * b < F.w && !full);
            }
            if (lane == 0) {
                sm.unfilled = (unsigned long long)bal[0] | ((unsigned long long)bal[1] << 32);
                sm.st[ST_LOST] += 1;
            }
        }
        __syncthreads();

        const int npatch = __popcll(sm.unfilled);
        if (wid == 0) fill_order(npatch);  // (read by warp 0 only)
        SK_PHASE(PH_STAGE);
        TraceRec* trace_base =
            (trace_on && F.trace) ? reinterpret_cast<TraceRec*>(F.trace) + (size_t)ent.z * 64 : nullptr;
        int step = 0;
        for (;;) {
            // Warp 0 alone runs the steps that stay in the base layer (Eq. (16), R3) back to
            // back; it stops at the first step that needs IDL and hands it to the CTA.
            if (wid == 0) {
                long long n_brl = 0, n_empty = 0, flops = 0, sum_ny = 0;
                int p = step < npatch ? sm.order[step] : 0;
                for (; step < npatch; ++step) {
                    // (the next patch of the order, read ahead of this step's chain of loads)
                    const int p_next = step + 1 < npatch ? sm.order[step + 1] : 0;
                    const int pa = p >> 3, pb = p & 7;
                    const int wr = kMB + 2 * pa - 2, wc = kMB + 2 * pb - 2;
                    const int pr = wr + 2, pc = wc + 2;
                    // lanes 0..3: pixel (lane >> 1, lane & 1) of the patch, its availability row
                    const unsigned long long prow = sm.av[pr + ((lane >> 1) & 1)];
                    const CtxStats cs = ctx_stats(sm, wr, wc, lane);
                    SK_PHASE(PH_CTX);
                    if (cs.ny > 0 && cs.phi > P.t_phi) {  // hand the step to the CTA
                        if (lane == 0) {
                            sm.hand.ymask = cs.ymask;
                            sm.hand.pa = pa;
                            sm.hand.pb = pb;
                            sm.hand.ny = cs.ny;
                            sm.hand.phi = cs.phi;
                            sm.hand.mean = cs.mean;
                        }
                        break;
                    }
                    const float xv = cs.ny == 0 ? 128.0f : cs.mean;
                    const int layer = cs.ny == 0 ? L_EMPTY : L_BRL;
                    if (lane < 4) {
                        float xw = fminf(fmaxf(xv, 0.0f), 255.0f);
                        if (force_on && trace_base) xw = trace_base[step].x[lane];  // verification hook
                        if (quant_on) xw = rintf(xw);
                        const int rr = pr + (lane >> 1), cc = pc + (lane & 1);
                        if (!((prow >> cc) & 1ull)) sm.S[rr * kReg + cc] = xw;  // lost pixels only
                    }
                    __syncwarp();
                    if (lane == 0) {
                        sm.av[pr] |= 3ull << pc;
                        sm.av[pr + 1] |= 3ull << pc;
                        sm.unfilled &= ~(1ull << p);
                        if (layer == L_EMPTY) ++n_empty;
                        else ++n_brl;
                        flops += 3ll * cs.ny;
                        sum_ny += cs.ny;
                    }
                    if (trace_base && lane == 0) {
                        TraceRec t;
                        t.mb = mb;
                        t.step = (int16_t)step;
                        t.patch = (int16_t)p;
                        t.layer = (int8_t)layer;
                        t.ring = 0;
                        t.beta_idx = -1;
                        t.n0 = 0;
                        t.ny = (int16_t)cs.ny;
                        t.m = 0;
                        t.phi = cs.phi;
                        t.log_nu = -INFINITY;
                        t.alpha = 0.0f;
                        t.eps_best = 0.0f;
                        for (int a = 0; a < 4; ++a) t.x[a] = fminf(fmaxf(xv, 0.0f), 255.0f);
                        for (int q = 0; q < 36; ++q) t.i0[q] = 0xffff;
                        trace_base[step] = t;
                    }
                    __syncwarp();
                    SK_PHASE(PH_BRL);
                    p = p_next;
                }
                if (lane == 0) {
                    sm.hand.step = step;
                    sm.st[ST_PATCH] += n_brl + n_empty;
                    sm.st[ST_BRL] += n_brl;
                    sm.st[ST_EMPTY] += n_empty;
                    sm.st[ST_FLOPS] += flops;
                    sm.st[ST_PATCH_NY] += sum_ny;
                }
            }
            __syncthreads();
            step = sm.hand.step;
            if (step >= npatch) break;

            StepCtx c;
            c.pa = sm.hand.pa;
            c.pb = sm.hand.pb;
            c.wr = kMB + 2 * c.pa - 2;
            c.wc = kMB + 2 * c.pb - 2;
            c.ymask = sm.hand.ymask;  // context: the window less the patch (from warp 0's ballots)
            c.ny = sm.hand.ny;
            c.phi = sm.hand.phi;
            c.mean = sm.hand.mean;

            float xhat[4];
            int layer;
            int ring = 0;
            float lognu = -INFINITY;
            long long evals = 0;
            if (trace_base && tid == 0) {
                sm.tr.beta_idx = -1;
                sm.tr.n0 = 0;
                sm.tr.alpha = 0.0f;
                sm.tr.eps_best = 0.0f;
                sm.tr.m = 0;
                for (int t = 0; t < 36; ++t) sm.tr.i0[t] = 0xffff;
            }
            {
                const IdlOut io = idl_step<MIXED, IDLTC>(P, c.wr, c.wc, c.ymask, c.ny, c.mean, mph);
                const int r = io.r;
                ring = io.ring;
                lognu = io.lognu;
                evals = io.evals;
#pragma unroll
                for (int a = 0; a < 4; ++a) xhat[a] = io.x[a];
                SK_PHASE(PH_IDL);
                if (tid == 0) {
                    sm.st[ST_IDL_EVALS] += evals;
                    sm.st[ST_IDL_NY] += evals * c.ny;
                    // per candidate: 3 Ny (difference, square, sum), exp, 5 weighted sums
                    sm.st[ST_FLOPS] += evals * (3ull * c.ny + 11ull);
                }
                if (r == 1) {
                    layer = L_IDL;
                } else if (r < 0) {
                    layer = L_NOCAND;
                    xhat[0] = xhat[1] = xhat[2] = xhat[3] = c.mean;
                } else {
                    layer = L_HQL;
                    __syncthreads();  // IDL slots -> HQL scratch
                    const HqlOut o = hql_step<MIXED>(P, c.wr, c.wc, c.ymask, c.ny, c.mean,
                                                     trace_base != nullptr, mph,
                                                     W.ubuf + (size_t)blockIdx.x * kUbufFloats);
                    mph = o.mph;
#pragma unroll
                    for (int a = 0; a < 4; ++a) xhat[a] = o.x[a];
                }
            }
            // R8: clip and write back
            if (tid == 0) {
                const int pr = c.wr + 2, pc = c.wc + 2;
#pragma unroll
                for (int a = 0; a < 4; ++a) xhat[a] = fminf(fmaxf(xhat[a], 0.0f), 255.0f);
                float xw[4] = {xhat[0], xhat[1], xhat[2], xhat[3]};
                if (force_on && trace_base) {  // verification hook: reference write-back
#pragma unroll
                    for (int a = 0; a < 4; ++a) xw[a] = trace_base[step].x[a];
                }
                if (quant_on) {
#pragma unroll
                    for (int a = 0; a < 4; ++a) xw[a] = rintf(xw[a]);
                }
#pragma unroll
                for (int a = 0; a < 4; ++a) {  // lost pixels only (received ones are available)
                    const int rr = pr + (a >> 1), cc = pc + (a & 1);
                    if (!((sm.av[rr] >> cc) & 1ull)) sm.S[rr * kReg + cc] = xw[a];
                }
                sm.av[pr] |= 3ull << pc;
                sm.av[pr + 1] |= 3ull << pc;
                sm.unfilled &= ~(1ull << (c.pa * 8 + c.pb));
                sm.st[ST_PATCH] += 1;
                sm.st[ST_FLOPS] += 3ull * c.ny;  // context gather, flatness, mean
                sm.st[ST_PATCH_NY] += c.ny;
                sm.st[layer == L_IDL ? ST_IDL : layer == L_HQL ? ST_HQL : ST_NOCAND] += 1;
                if (layer == L_IDL) sm.st[ST_RING0 + min(ring, 15)] += 1;
                if (trace_base) {
                    TraceRec& t = sm.tr;
                    t.mb = mb;
                    t.step = (int16_t)step;
                    t.patch = (int16_t)(c.pa * 8 + c.pb);
                    t.layer = (int8_t)layer;
                    t.ring = (int8_t)ring;
                    t.ny = (int16_t)c.ny;
                    t.phi = c.phi;
                    t.log_nu = lognu;
                    for (int a = 0; a < 4; ++a) t.x[a] = xhat[a];
                    trace_base[step] = t;
                }
            }
            __syncthreads();
            SK_PHASE(PH_WB);
            ++step;
        }

        // publish: unrounded values for dependants, rounded / FP32 outputs
        for (int i = tid; i < 256; i += kThreads) {
            const int r = i >> 4, cc = i & 15;
            const float v = sm.S[(kMB + r) * kReg + kMB + cc];
            W.vals[(size_t)e * 256 + i] = v;
            const int fy = mby * kMB + r, fx = mbx * kMB + cc;
            if (fy < F.h && fx < F.w) {
                F.out[(size_t)fy * F.out_pitch + fx] = (uint8_t)__float2int_rn(v);
                if (F.out_f32) F.out_f32[(size_t)fy * F.out_f32_pitch + fx] = v;
            }
        }
        __threadfence();
        __syncthreads();
        if (tid == 0) {
            st_release(&W.done[e], 1u);
            if (P.concealed_is_support) release_dependants(W, F, mb);
        }
        SK_PHASE(PH_PUB);
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (MIXED && wid == 0) tc::tmem_dealloc(sm.tmem_base, kTmemCols<MIXED>);
    if (tid == 0 && sm.mma_err) atomicExch(&W.counters[2], 6);
    if (tid == 0) sm.st[ST_T_LAST] = globaltimer_ns();
    __syncthreads();
    for (int i = tid; i < kNStats; i += kThreads) {
        if (i == ST_T_FIRST_INV || i == ST_T_LAST) atomicMax(&W.stats[i], sm.st[i]);
        else if (sm.st[i]) atomicAdd(&W.stats[i], sm.st[i]);
    }
}

// ------------------------------------------------------------------------------------
// Block flags of per-pixel loss masks: a block is lost iff it holds a lost pixel.  One CTA
// per frame, one warp per block (lane: half a row of the block).  Frames given block flags
// are skipped.  flags: the derived flags of all frames, at each frame's mb_base.
__global__ void __launch_bounds__(kThreads) px_block_flags_kernel(const __grid_constant__ WorkDev W,
                                                                   uint8_t* flags) {
    const FrameDev& F = W.frames[blockIdx.x];
    if (!F.px_lost) return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nmb = F.mbw * F.mbh;
    for (int mb = wid; mb < nmb; mb += kWarps) {
        const int by = mb / F.mbw, bx = mb - by * F.mbw;
        const int y = by * kMB + (lane >> 1), x0 = bx * kMB + (lane & 1) * 8;
        bool any = false;
        if (y < F.h) {
            const uint8_t* row = F.px_lost + (size_t)y * F.px_pitch;
#pragma unroll
            for (int i = 0; i < 8; ++i)
                if (x0 + i < F.w && row[x0 + i] != 0) any = true;
        }
        const bool lost = __any_sync(0xffffffffu, any);
        if (lane == 0) flags[F.mb_base + mb] = lost ? 1 : 0;
    }
}

// ------------------------------------------------------------------------------------
// Work queue.  A lost block depends on its lost neighbours earlier in raster order (left,
// top-left, top, top-right) when concealed pixels are support.  The blocks of a call are
// grouped into buckets by their height, the length of the longest chain of blocks that
// depend on them (0 for a block nothing waits for); bucket key = nbk - 2 - height, so low
// keys hold the blocks that head the longest chains.  Blocks with no lost neighbour at all
// take the last bucket, nbk - 1, after every block of a loss cluster: a block's cost is not
// known before it runs (it is set by how many of its steps reach HQL), and run this way the
// clusters' blocks, which carry the chains and on average more HQL steps, do not end up
// behind the isolated ones at the end of the call, where one expensive block left alone
// holds the whole call.  A block becomes ready when its last dependency is done and is
// then published in its bucket; a free CTA claims a ready block of the lowest live key
// (highest height first: list scheduling by critical path).  A CTA only ever claims ready
// blocks, so no CTA holds an SM while it waits for a dependency.

constexpr int kIsolated = -2;  // height_of_mb of a lost block with no lost neighbour

__device__ __forceinline__ int bucket_key(const WorkDev& W, int h) {
    return h == kIsolated ? W.nbk - 1 : max(0, W.nbk - 2 - h);
}

struct SegFV {
    int f;  // a segment starts inside the combined range
    int v;  // running maximum since the last segment start
};

__device__ __forceinline__ SegFV seg_combine(SegFV a, SegFV b) {
    return {a.f | b.f, b.f ? b.v : max(a.v, b.v)};
}

// inclusive segmented max-scan over the CTA (one element per thread, thread order)
__device__ __forceinline__ SegFV block_seg_scan(SegFV x, SegFV* sh /*[kWarps]*/) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        SegFV y;
        y.f = __shfl_up_sync(0xffffffffu, x.f, o);
        y.v = __shfl_up_sync(0xffffffffu, x.v, o);
        if (lane >= o) x = seg_combine(y, x);
    }
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    if (wid > 0) {
        SegFV pre = sh[0];
        for (int w = 1; w < wid; ++w) pre = seg_combine(pre, sh[w]);
        x = seg_combine(pre, x);
    }
    __syncthreads();
    return x;
}

constexpr int kLevelNeg = -(1 << 29);

// one CTA per frame: height of every lost block, rows from the bottom up.  The dependants
// of (y, x) are the lost blocks (y, x+1) and (y+1, x-1 .. x+1).  Within a row a run of lost
// blocks chains through the right neighbour, so with the mirrored column x' = mbw-1-x,
// height[x'] = x' + max over the run up to x' of (down[k'] - k'), down = max(0, 1 + height
// of the lost blocks below): a segmented max-scan.  Also counts the blocks of each bucket.
__global__ void __launch_bounds__(kThreads) queue_heights_kernel(WorkDev W, int support) {
    __shared__ SegFV sh[kWarps];
    __shared__ int carry_s;
    __shared__ int cnt_s;
    const int f = blockIdx.x, tid = threadIdx.x;
    const FrameDev& F = W.frames[f];
    int* hgt = W.height_of_mb + F.mb_base;
    if (tid == 0) cnt_s = 0;
    int cnt = 0;
    for (int y = F.mbh - 1; y >= 0; --y) {
        if (tid == 0) carry_s = kLevelNeg;
        __syncthreads();
        for (int x0 = 0; x0 < F.mbw; x0 += kThreads) {
            const int xm = x0 + tid, x = F.mbw - 1 - xm;
            const bool in = xm < F.mbw;
            const bool lost = in && F.lost[y * F.mbw + x] != 0;
            bool isolated = lost;
            if (lost) {
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        const int yy = y + dy, xx = x + dx;
                        if ((dy || dx) && yy >= 0 && yy < F.mbh && xx >= 0 && xx < F.mbw &&
                            F.lost[yy * F.mbw + xx])
                            isolated = false;
                    }
            }
            int down = 0;
            if (lost && support && y + 1 < F.mbh) {
                for (int dx = -1; dx <= 1; ++dx) {
                    const int xx = x + dx;
                    if (xx >= 0 && xx < F.mbw && F.lost[(y + 1) * F.mbw + xx])
                        down = max(down, hgt[(y + 1) * F.mbw + xx] + 1);
                }
            }
            const bool right_lost = in && x + 1 < F.mbw && F.lost[y * F.mbw + x + 1] != 0;
            SegFV e;
            e.f = (!lost || !right_lost || !support) ? 1 : 0;
            e.v = lost ? down - xm : kLevelNeg;
            // a run continuing from the previous chunk starts without a head in this chunk
            if (tid == 0 && x0 > 0 && lost && right_lost && support) e.f = 0;
            SegFV r = block_seg_scan(e, sh);
            const int carry = carry_s;
            if (!r.f) r.v = max(r.v, carry);
            if (lost) {
                int h = support ? xm + r.v : 0;
                if (h < 0 || h >= W.nbk) {  // cannot happen (a chain has at most nbk blocks)
                    atomicExch(&W.counters[2], 7);
                    h = min(max(h, 0), W.nbk - 1);
                }
                if (isolated) h = kIsolated;  // (height 0: nothing depends on it)
                hgt[y * F.mbw + x] = h;
                atomicAdd(&W.bk_off[bucket_key(W, h)], 1);
                ++cnt;
            } else if (in) {
                hgt[y * F.mbw + x] = -1;
            }
            __syncthreads();
            if (tid == kThreads - 1) carry_s = (lost && support) ? r.v : kLevelNeg;
            __syncthreads();
        }
    }
    atomicAdd(&cnt_s, cnt);
    __syncthreads();
    if (tid == 0) atomicAdd(&W.counters[0], cnt_s);
}

// one CTA: exclusive scan of the bucket sizes into first-entry offsets; the first non-empty
// bucket starts the claim scan
__global__ void __launch_bounds__(kThreads) queue_offsets_kernel(WorkDev W) {
    __shared__ int scan[kWarps + 1];
    __shared__ int first_s;
    if (threadIdx.x == 0) first_s = W.nbk;
    __syncthreads();
    int run = 0;
    for (int l0 = 0; l0 < W.nbk; l0 += kThreads) {
        const int l = l0 + threadIdx.x;
        const int v = l < W.nbk ? W.bk_off[l] : 0;
        if (v > 0) atomicMin(&first_s, l);
        int tot;
        const int ex = block_exscan(v, scan, &tot) + run;
        if (l < W.nbk) W.bk_off[l] = ex;
        run += tot;
    }
    __syncthreads();
    if (threadIdx.x == 0) W.counters[3] = first_s;
}

// one CTA per frame: every lost block takes the next entry of its bucket and counts its
// dependencies; blocks without any are published as ready.  The rank among the frame's
// lost blocks in raster order indexes its trace records.
__global__ void __launch_bounds__(kThreads) queue_fill_kernel(WorkDev W, int support) {
    __shared__ int scan[kWarps + 1];
    const int f = blockIdx.x;
    const FrameDev& F = W.frames[f];
    const int nmb = F.mbw * F.mbh;
    int run = 0;
    for (int t0 = 0; t0 < nmb; t0 += kThreads) {
        const int i = t0 + threadIdx.x;
        const int lost = (i < nmb) ? (F.lost[i] != 0) : 0;
        int tot;
        const int rank = block_exscan(lost, scan, &tot) + run;
        if (i < nmb) {
            if (lost) {
                const int key = bucket_key(W, W.height_of_mb[F.mb_base + i]);
                const int e = W.bk_off[key] + atomicAdd(&W.bk_cnt[key], 1);
                W.entry_of_mb[F.mb_base + i] = e;
                W.entries[e] = make_int4(f, i, rank, key);
                W.done[e] = 0u;
                int ndep = 0;
                if (support) {
                    const int y = i / F.mbw, x = i - y * F.mbw;
                    if (x > 0 && F.lost[i - 1]) ++ndep;
                    if (y > 0) {
                        for (int dx = -1; dx <= 1; ++dx) {
                            const int xx = x + dx;
                            if (xx >= 0 && xx < F.mbw && F.lost[i - F.mbw + dx]) ++ndep;
                        }
                    }
                }
                W.rem[e] = ndep;
                if (ndep == 0) {
                    const int k = atomicAdd(&W.bk_tail[key], 1);
                    W.slots[W.bk_off[key] + k] = e;
                }
            } else {
                W.entry_of_mb[F.mb_base + i] = -1;
            }
        }
        run += tot;
    }
}

}  // namespace sk

namespace sk {
static_assert(sizeof(Smem) <= 113 * 1024, "two CTAs per SM");
static_assert(offsetof(Hql, mx) % 16 == 0 && sizeof(Hql::mx) == 4 * 128 * 64 * 2, "tensor-core tiles");
static_assert((offsetof(Smem, hql) + offsetof(Hql, mx)) % 128 == 0, "tensor-core tiles on 128-byte lines");
static_assert(kReg % kWarps == 0, "rows of the support region per warp");
static_assert(offsetof(Hql, cand) % 16 == 0 && offsetof(Hql, d) % 16 == 0 && offsetof(Hql, off) % 16 == 0,
              "16-byte loads of candidate indices, distances and context offsets");
static_assert(offsetof(Hql, Z) % 16 == 0 && offsetof(Hql, Linv) % 16 == 0 && offsetof(Hql, G) % 16 == 0 &&
                  offsetof(Hql, ys) % 16 == 0 && offsetof(Smem, hql) % 16 == 0,
              "float4 operands");
}  // namespace sk

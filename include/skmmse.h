/*
 * skmmse.h -- C ABI of the GB300 (sm_103a) implementation of scalable kernel-based
 * MMSE (SK-MMSE) spatial error concealment, Koloda, Seiler, Peinado, Kaup,
 * arXiv 2205.11226.
 *
 * Problem statement (Sec. II): a frame R = L u S holds missing pixels L (here: whole
 * 16x16 blocks flagged in a block-loss map) and available pixels S.  Each lost block is
 * filled 2x2 patch by 2x2 patch from its border inwards; every patch x0 is estimated
 * from its context y0 (the available pixels of the 6x6 window centred on x0) and from
 * candidates z_j = (x_j, y_j) with the same spatial configuration found in the 8
 * neighbouring blocks, by one of three layers chosen per patch by a profile (Sec. V):
 *   BRL  context mean, Eq. (16), when the flatness phi = max(y0) - min(y0) <= T_phi
 *        (Eq. (17));
 *   IDL  exponential weights with scalar bandwidth sigma^2 * Ny over a support area
 *        growing from x0, Eq. (15), accepted when the normaliser nu >= T_nu (Eq. (18));
 *   HQL  full K-MMSE with sample-covariance bandwidth and beta/alpha fitting,
 *        Eq. (13) with Eqs. (3)-(12).
 * A reconstructed patch joins the support (end of Sec. III).
 *
 * Conventions for every entry point:
 *   - Pointers named d_* and the pointers inside skmmse_frame are DEVICE memory owned by
 *     the caller; h_* pointers are host memory owned by the caller.  The library never
 *     frees caller memory.
 *   - Frames are 8-bit luma, `height` rows of `pitch` bytes; width and height must be
 *     even and positive.  The block-loss map has ceil(height/16) rows of ceil(width/16)
 *     bytes, non-zero = lost.  Partial blocks at the right/bottom edge conceal only their
 *     in-frame pixels.  Input values of lost pixels are never read.
 *   - Work is enqueued asynchronously on `stream` (a cudaStream_t, NULL = legacy default
 *     stream).  Argument errors are returned synchronously and enqueue nothing; device
 *     errors (a dependency wait that gave up) are reported by skmmse_read_stats().
 *     Passing a non-NULL h_stats makes the call synchronous on `stream`.
 *   - A context owns device scratch memory (work queue, dependency flags, the unrounded
 *     values of concealed blocks, counters), grown on demand with cudaMalloc and freed by
 *     skmmse_destroy().  Calls sharing a context must be ordered on one stream; use one
 *     context per concurrently running stream.
 *   - No exception crosses this ABI.  All functions are thread-compatible, not
 *     thread-safe on one context.
 */
#ifndef SKMMSE_H_
#define SKMMSE_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SKMMSE_ABI_VERSION 3

typedef enum {
    SKMMSE_OK = 0,
    SKMMSE_ERR_ARG = 1,         /* NULL pointer, bad parameter value */
    SKMMSE_ERR_SHAPE = 2,       /* odd or non-positive size, pitch < width, too many frames */
    SKMMSE_ERR_ALIGN = 3,       /* pointer or pitch alignment not supported */
    SKMMSE_ERR_NOMEM = 4,       /* scratch allocation failed */
    SKMMSE_ERR_CUDA = 5,        /* a CUDA runtime call failed */
    SKMMSE_ERR_TIMEOUT = 6,     /* a wait on the device gave up, or the work queue found an
                                   inconsistent block graph (device error word) */
    SKMMSE_ERR_UNSUPPORTED = 7, /* requested precision or flag not built */
    SKMMSE_ERR_TOO_LARGE = 8    /* frame larger than the static scratch of
                                   skmmse_conceal_noalloc (SKMMSE_NOALLOC_MAX_MBS blocks) */
} skmmse_status;

/* Arithmetic of the HQL contractions (Eqs. (7)-(10)).  FP32: every step in FP32 on the
   CUDA cores (covariance with exact integer parts, factorisation in double-float).  The
   mixed modes run the covariance, the whitened (Mahalanobis) distances and the beta-grid
   sums on tcgen05 tensor cores with FP32 accumulation: integer parts of the covariance
   exactly, every other operand split into a high and a low 16-bit half.  Exponentials,
   normalisations, the IDL layer and the leave-one-out pass stay FP32.  Teacher-forced per
   step against an FP64 reference: FP16 within ~2e-3 gray, BF16 within ~4e-2 gray. */
typedef enum { SKMMSE_FP32 = 0, SKMMSE_MIXED_BF16 = 1, SKMMSE_MIXED_FP16 = 2 } skmmse_precision;

/* Profiles of Table I (T_phi, T_nu): express (20, 0.01), efficient (20, 0.1),
   excellent (20, 100). */
typedef enum { SKMMSE_EXPRESS = 0, SKMMSE_EFFICIENT = 1, SKMMSE_EXCELLENT = 2 } skmmse_profile;

/* flags */
#define SKMMSE_FLAG_TRACE 1u   /* write per-patch decision records (skmmse_frame.trace) */
/* Verification hook (requires SKMMSE_FLAG_TRACE): the trace buffer is read before it is
   written; its x[4] fields hold reference estimates, which the kernel writes back into
   the support instead of its own estimates ("teacher forcing").  The records written
   carry the kernel's own estimates, so each step can be compared with a reference on
   identical inputs.  Outputs then hold the reference values.  Not for production use. */
#define SKMMSE_FLAG_FORCE 2u
/* In-loop 8-bit quantisation: every estimate is written back into the support rounded to
   the nearest integer (ties to even), as a decoder that keeps 8-bit frames does; the
   reading of the end of Sec. III that keeps unrounded values is the default.  Later
   templates then hold integers only.  Trace records keep the unrounded estimate. */
#define SKMMSE_FLAG_QUANTIZE 4u
/* Test hook for failure detection: a CTA that finds no ready block gives up after 64
   polls without progress instead of ~2^25 (about 9 s).  On a workload with dependency
   chains idle CTAs then give up while others still work: the call still conceals every
   block (the working CTAs take the rest), sets the device error word and returns
   SKMMSE_ERR_TIMEOUT, and the context stays usable.  Not for production use. */
#define SKMMSE_FLAG_SHORT_WAITS 8u
/* IDL distances on tensor cores (mixed precision only; ignored in FP32): when a patch's
   first ring does not reach T_nu, the distances of Eq. (15) for all 43 x 43 window
   positions are formed in one pass of Toeplitz products on tcgen05 (per window row r, the
   region's rows r.. against the template row, high and low 16-bit halves, and the squared
   region against the context mask), and the later rings read them.  Exact for integer
   templates and windows; otherwise within the split's precision.  Off by default. */
#define SKMMSE_FLAG_IDL_TC 16u

typedef struct {
    float t_phi;        /* flatness threshold T_phi, Eq. (17) / Table I; BRL iff phi <= T_phi */
    float t_nu;         /* normalisation threshold T_nu, Eq. (18) / Table I; must be > 0 */
    float sigma2;       /* IDL aperture sigma^2, Eq. (14); 10 in the paper (Sec. IV-B) */
    int ring_step;      /* IDL support growth: ring k holds candidate patches at Chebyshev
                           distance in ((k-1)*ring_step, k*ring_step] from x0; >= 1 */
    float ridge_rel;    /* HQL: C_YY += (ridge_rel * trace(C_YY)/Ny + 1e-6) I; >= 0 */
    int beta_kmin;      /* HQL beta grid: beta = 2^(k/2), k = beta_kmin..beta_kmax */
    int beta_kmax;      /*   (at most 32 grid values) */
    float beta_tie_rel; /* HQL: beta* = smallest grid beta with eps_y <= (1+tie) min eps_y */
    int concealed_is_support; /* 1: blocks concealed earlier in raster order are support */
    int precision;      /* skmmse_precision */
    unsigned flags;     /* SKMMSE_FLAG_* */
} skmmse_params;

/* One frame of a batch.  All pointers are device memory.  `out` may equal `frame`
   (in-place).  `out_f32` (nullable) receives unrounded values: every pixel of a lost
   block in the frame; pixels outside lost blocks are not written.  `trace` (nullable,
   used with SKMMSE_FLAG_TRACE) holds n_lost*64 skmmse_trace_rec, indexed by
   [rank of the block among the frame's lost blocks in raster order][fill step].

   The loss is given by exactly one of two masks (the other NULL):
   - mb_lost: ceil(height/16) x ceil(width/16) bytes, 1 = the whole 16x16 block is lost
     (the loss the paper's experiments use);
   - px_lost: `height` rows of `px_pitch` bytes, 1 = the pixel is lost: an arbitrarily
     shaped loss (Sec. II notes the method extends to any shape).  A block holding a lost
     pixel is a lost block (the unit of work, with the same dependencies); received
     pixels are support wherever they lie; the 2x2 patches holding a lost pixel are
     filled in the fill order; a patch's own pixels are never context, and only its lost
     pixels take the estimate, so received pixels leave the call unchanged.  A px_lost
     that loses whole blocks gives the mb_lost result bit for bit. */
typedef struct {
    const uint8_t* frame;
    int width, height, pitch;
    const uint8_t* mb_lost;
    uint8_t* out;
    int out_pitch;
    float* out_f32;
    int out_f32_pitch;  /* in floats */
    void* trace;
    const uint8_t* px_lost;
    int px_pitch;       /* in bytes, >= width when px_lost is given */
    int reserved;       /* 0 */
} skmmse_frame;

/* Per-patch decision record (SKMMSE_FLAG_TRACE). */
typedef struct {
    int32_t mb;         /* block raster index in its frame */
    int16_t step;       /* fill step inside the block */
    int16_t patch;      /* patch index a*8+b (a = patch row, b = patch column) */
    int8_t layer;       /* 0 Ny=0 fill, 1 BRL, 2 IDL, 3 HQL, 4 BRL (no candidate) */
    int8_t ring;        /* IDL: accepted ring; otherwise rings evaluated */
    int8_t beta_idx;    /* HQL: index of beta* in the grid, else -1 */
    int8_t n0;          /* HQL: |I0| */
    int16_t ny;         /* context size */
    int16_t m;          /* candidates in the whole support (when enumerated) */
    float phi;          /* flatness */
    float log_nu;       /* log nu after the last ring evaluated */
    float alpha;        /* HQL alpha after clamping */
    float eps_best;     /* HQL eps_y(beta*) */
    float x[4];         /* estimate after clipping */
    uint16_t i0[36];    /* HQL I0 as window indices wu*43+wv (43 positions per axis in the
                           48x48 support region), ascending; unused entries 0xffff */
} skmmse_trace_rec;

/* Counters of one call (summed over the batch). */
typedef struct {
    long long n_lost_mbs;
    long long n_patches, n_empty, n_brl, n_idl, n_hql, n_brl_nocand;
    long long idl_ring_hist[16];
    long long idl_cand_evals;   /* IDL candidate distance evaluations */
    long long idl_ny_evals;     /* sum of Ny over those evaluations */
    long long hql_cands;        /* sum of M over HQL patches */
    long long hql_ny_cands;     /* sum of M*Ny over HQL patches */
    long long hql_i0_cands;     /* sum of |I0|*M over HQL patches */
    long long alg_flops;        /* algorithmic FP32 operations of the call, an exp counting as
                                   one: per patch 3 Ny (context gather, flatness, mean); per IDL
                                   candidate 3 Ny + 11 (distance, exp, five weighted sums); per
                                   HQL patch with M candidates, Ny context values, |G| beta
                                   values and |I0| = n0 members
                                   M (Ny (Ny+1) + 8 Ny + 2 (Ny+4))     covariance C_YY, C_XY, sums
                                   + M (Ny (Ny+1) + 2 Ny)              whitening and distance
                                   + |G| M (2 (Ny+5) + 3)              beta grid
                                   + n0 M (3 Ny + 2 (Ny+5) + 3)        leave-one-out */
    long long hql_ny2_cands;    /* sum of M*Ny^2 over HQL patches */
    long long hql_ny3;          /* sum of Ny^3 over HQL patches (the factorisation's order) */
    long long hql_i0_ny_cands;  /* sum of |I0|*M*Ny over HQL patches */
    long long patch_ny;         /* sum of Ny over all patches */
    long long mma_flops;        /* tensor-core operations issued (2 M N K per tcgen05.mma), mixed
                                   precision only */
    long long t_first_inv_ns;   /* ~(start of the concealment kernel's first CTA), global timer */
    long long t_last_ns;        /* end of its last CTA, global timer (ns): the launch's resident
                                   interval is [~t_first_inv_ns, t_last_ns] */
    long long n_beta;           /* beta grid size of the call */
    int error;                  /* 0; else the device error word: 6 a wait gave up, 7 the
                                   work queue met an impossible chain height */
    int pad;
} skmmse_stats;

typedef struct skmmse_context skmmse_context;

/* Library and ABI version (SKMMSE_ABI_VERSION). */
int skmmse_abi_version(void);

/* Size in bytes of skmmse_trace_rec / skmmse_stats / skmmse_params / skmmse_frame /
   skmmse_config (lets a binding check its struct layout); -1 for other values. */
int skmmse_struct_size(int which /* 0 trace, 1 stats, 2 params, 3 frame, 4 config */);

/* Human-readable status. Never NULL. */
const char* skmmse_status_str(skmmse_status s);

/* Fill *p with a Table I profile, sigma^2 = 10 and the default readings of the
   unstated parts: ring_step 4, ridge_rel 1e-3, beta grid k = -8..16, beta_tie_rel 1e-3,
   concealed_is_support 1, FP32, no flags.  Unknown profile -> efficient. */
void skmmse_params_preset(skmmse_params* p, int profile);

/* Create a context on the current CUDA device.  Returns SKMMSE_ERR_ARG for ctx == NULL,
   SKMMSE_ERR_CUDA if no device is usable. */
skmmse_status skmmse_create(skmmse_context** ctx);

/* Release the context's scratch memory (synchronises its last stream). NULL is a no-op. */
void skmmse_destroy(skmmse_context* ctx);

/* Conceal all lost blocks of one frame: the frame's received pixels are copied to d_out,
   and each lost block is filled by the layered SK-MMSE estimate (Secs. II-V).
   d_out_f32 (nullable): unrounded values of lost pixels, pitch = width floats.
   The rounded output is round-half-even of the clipped estimate. */
skmmse_status skmmse_conceal(skmmse_context* ctx, const uint8_t* d_frame, int width,
                             int height, int pitch, const uint8_t* d_mb_lost,
                             const skmmse_params* p, uint8_t* d_out, int out_pitch,
                             float* d_out_f32, skmmse_stats* h_stats, void* stream);

/* The same for an arbitrarily shaped loss: d_px_lost holds `height` rows of `px_pitch`
   bytes, 1 = lost pixel (see skmmse_frame.px_lost).  d_out_f32 (nullable): unrounded
   values of every pixel of the blocks holding a lost pixel (received ones unchanged). */
skmmse_status skmmse_conceal_px(skmmse_context* ctx, const uint8_t* d_frame, int width,
                                int height, int pitch, const uint8_t* d_px_lost, int px_pitch,
                                const skmmse_params* p, uint8_t* d_out, int out_pitch,
                                float* d_out_f32, skmmse_stats* h_stats, void* stream);

/* Conceal n frames of any sizes in one persistent launch (one work queue over all lost
   blocks of all frames; a block is claimed once its dependencies are done, the block
   heading the longest remaining chain first).  h_frames is a host array of n descriptors
   (1 <= n <= 65536). */
skmmse_status skmmse_conceal_batch(skmmse_context* ctx, const skmmse_frame* h_frames, int n,
                                   const skmmse_params* p, skmmse_stats* h_stats,
                                   void* stream);

/* Synchronise `stream` and copy the counters of the context's last call into *h_stats.
   Returns SKMMSE_ERR_TIMEOUT if a dependency wait gave up during that call. */
skmmse_status skmmse_read_stats(skmmse_context* ctx, skmmse_stats* h_stats, void* stream);

/* A batch call recorded as a CUDA graph on fixed frame buffers: the received-pixel copies,
   the queue construction and the persistent concealment kernel.  The frame descriptors and
   TMA maps are uploaded once, synchronously, into device memory owned by the graph (which
   also owns its scratch); each launch conceals what the frame buffers hold when it runs,
   asynchronously on `stream`.  Launches of one graph must be ordered on one stream. */
typedef struct skmmse_graph skmmse_graph;
skmmse_status skmmse_graph_create(skmmse_context* ctx, const skmmse_frame* h_frames, int n,
                                  const skmmse_params* p, skmmse_graph** out);
skmmse_status skmmse_graph_launch(skmmse_graph* g, void* stream);
/* Synchronise `stream` and return the counters of the graph's last launch. */
skmmse_status skmmse_graph_read_stats(skmmse_graph* g, skmmse_stats* h_stats, void* stream);
void skmmse_graph_destroy(skmmse_graph* g);

/* Launch configuration of the concealment kernel (the paper has no counterpart; none of these
   changes a result: every block's arithmetic runs in one CTA in a fixed order, and the
   tensor-core passes accumulate the same 16-candidate slices in the same order whatever
   the tile):
     ctas_per_sm  persistent CTAs per SM, 1 .. the occupancy maximum (2), 0 = the maximum;
                  fewer CTAs give each block more of its SM and shorten dependency chains,
                  more run more blocks at once;
     tile_cov     candidates per chunk of the HQL covariance pass (the MMAs' K, Eq. (8)):
                  32 or 64;
     tile_dist    candidates per tile of the whitened-distance pass (the MMA's M, Eq. (6)
                  with C_YY): 64 or 128.
   The tiles apply to the mixed precisions; the FP32 path ignores them. */
typedef struct {
    int ctas_per_sm;
    int tile_cov;
    int tile_dist;
} skmmse_config;
#define SKMMSE_TUNE_MAX_OPTIONS 8

/* Autotuner: conceals the given batch `reps` times (plus one warm-up) for every
   configuration (CTAs per SM the occupancy allows x tile_cov {32, 64} x tile_dist {64, 128};
   CTAs per SM only in FP32), and keeps the fastest for the batch's shape class in the
   context: the calls and graphs of that class use it.  A shape class is the precision,
   profile thresholds and support rule of p, and the number, sizes and mask kinds of the
   frames (loss maps live in device memory and are not read).  Up to 64 classes are kept
   (the oldest is replaced).  h_options / h_ms (nullable, SKMMSE_TUNE_MAX_OPTIONS entries)
   receive the configurations timed and their mean device milliseconds, *h_n_options their
   number and *h_best the index of the fastest (each nullable).  The outputs of the batch are
   written by every run.  Synchronous. */
skmmse_status skmmse_autotune(skmmse_context* ctx, const skmmse_frame* h_frames, int n,
                              const skmmse_params* p, int reps, void* stream,
                              skmmse_config* h_options, float* h_ms, int* h_n_options,
                              int* h_best);
/* The configuration used for shape classes the autotuner has not timed (initially
   {0, 64, 64}).  Values outside the ranges above return SKMMSE_ERR_ARG. */
skmmse_status skmmse_set_config(skmmse_context* ctx, const skmmse_config* cfg);
/* The configuration a call with these frames and parameters would use. */
skmmse_status skmmse_get_config(skmmse_context* ctx, const skmmse_frame* h_frames, int n,
                                const skmmse_params* p, skmmse_config* out);
/* Set the default's persistent CTAs per SM directly (0 = occupancy maximum). */
skmmse_status skmmse_set_ctas_per_sm(skmmse_context* ctx, int ctas_per_sm);

/* Largest frame, in 16x16 blocks (partial edge blocks included), that
   skmmse_conceal_noalloc accepts: 8192 covers 1920x1080 (120 x 68 = 8160 blocks). */
#define SKMMSE_NOALLOC_MAX_MBS 8192
/* Persistent CTAs skmmse_conceal_noalloc launches at most (each keeps the whitened vectors
   of its current HQL step, 1849 x 32 floats, in the static scratch). */
#define SKMMSE_NOALLOC_MAX_CTAS 128
/* Bytes of the static device array behind skmmse_conceal_noalloc (about 39.1 MB). */
#define SKMMSE_NOALLOC_SCRATCH_BYTES 39109888

/* skmmse_conceal_noalloc: the same concealment as skmmse_conceal for one frame, for callers
   that cannot allocate device memory -- for example code running inside a memory pool or
   an allocator hook, under a strict device-memory budget, or anywhere a cudaMalloc would
   synchronise or fail.  The paper has no counterpart; this is an interface convenience.
   It calls no cudaMalloc, cudaFree, cudaMallocHost or allocating library routine.  Its
   scratch (work queue, dependency flags, per-block values, counters, and the whitened
   vectors of the HQL step each persistent CTA is on) is one static device array of
   SKMMSE_NOALLOC_SCRATCH_BYTES (about 39.1 MB), sized for SKMMSE_NOALLOC_MAX_MBS blocks and
   SKMMSE_NOALLOC_MAX_CTAS persistent CTAs; every GPU that loads the library holds it until
   the process exits.  Larger frames return SKMMSE_ERR_TOO_LARGE.  The results are those of
   skmmse_conceal (the number of persistent CTAs does not change them).
   The first call on a device (and the first after the device's primary context was
   replaced, e.g. by cudaDeviceReset) looks up the array's device address and sets kernel
   attributes for that device: make it before any stream capture on that device.  All
   calls share the one array and it keeps the last call's contents: calls that may overlap
   on the GPU (different streams, or host threads without ordering) race; order them on one
   stream.  Arguments as skmmse_conceal (whole-block loss only); p->flags may hold
   SKMMSE_FLAG_QUANTIZE only (no trace).  h_stats (nullable) makes the call synchronous
   and returns the counters.  Errors found on the device (a wait that gave up, status 6)
   are reported only through h_stats: a call without h_stats cannot learn of them. */
skmmse_status skmmse_conceal_noalloc(const uint8_t* d_frame, int width, int height, int pitch,
                                     const uint8_t* d_mb_lost, const skmmse_params* p,
                                     uint8_t* d_out, int out_pitch, float* d_out_f32,
                                     skmmse_stats* h_stats, void* stream);

/* Diagnostic: per-phase SM clock cycles of the context's last call, summed over CTAs
   (thread 0's view, barrier waits included): 0 staging, 1 patch selection and context,
   2 BRL, 3 IDL, 4 HQL candidate list, 5 covariance, 6 factorisation, 7 distances,
   8 beta grid, 9 I0, 10 leave-one-out pass, 11 HQL estimate, 12 write-back, 13 publish.
   All zero unless the library was built with -DSKMMSE_PHASE_CLOCKS.  Synchronises. */
skmmse_status skmmse_read_phase_clocks(skmmse_context* ctx, long long* h_clocks16, void* stream);

/* Diagnostic (the paper has no counterpart): measured throughput of the current device's
   FP32 FMA pipe (*h_fma_tflops, TFLOP/s, 2 FLOP per FMA) and of its exp2 unit
   (*h_ex2_per_s, ex2.approx per second), from two short saturating kernels (8 CTAs of 256
   threads per SM, 8 independent chains per thread) timed with CUDA events on `stream`.
   The benchmark divides by them for its ALU and exp roofline fractions.  Allocates and
   frees a small device buffer; synchronises. */
skmmse_status skmmse_probe_peaks(double* h_fma_tflops, double* h_ex2_per_s, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SKMMSE_H_ */

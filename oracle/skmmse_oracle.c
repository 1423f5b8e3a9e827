/*
 * SK-MMSE spatial error concealment: plain FP64 CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct statement of
 * what the CUDA path computes.  Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark load it.  It shares no code, header, table or constant with
 * the CUDA library, and nothing in the product path calls it.
 *
 * Paper: Koloda, Seiler, Peinado, Kaup, "Scalable Kernel-Based Minimum Mean Square
 * Error Estimator for Accelerated Image Error Concealment" (arXiv 2205.11226).
 *
 * Method summary with the passages each part follows:
 *   - Sec. II: a missing vector x0 (a 2x2 patch) is estimated from its context y0,
 *     the available pixels of the 6x6 neighbourhood centred on x0; candidates
 *     z_j = (x_j, y_j) are all vectors with the same spatial configuration that can
 *     be built from available pixels of the support area S = the 8 blocks around the
 *     lost 16x16 block.  Lost blocks are filled from the outer border towards the
 *     centre; a reconstructed patch joins S (end of Sec. III).
 *   - Sec. IV-C, Eq. (16): BRL, the mean of y0.
 *   - Sec. IV-B, Eqs. (14)-(15): IDL, exponential weights with scalar bandwidth
 *     sigma^2 * Ny over a support area growing from the current patch.
 *   - Sec. IV-A, Eq. (13) with Sec. III, Eqs. (3)-(12): HQL, full K-MMSE.
 *   - Sec. V, Eqs. (17)-(18), Table I: the profile decision.
 *
 * Readings where the paper is silent or garbled (each is a parameter or rule here):
 *   R1  lost blocks are processed in raster order; pixels of blocks concealed earlier
 *       are support (concealed_is_support=1) or not (0).
 *   R2  fill order: among unfilled patches, the one with the most available pixels
 *       in its 6x6 window; ties to the lowest raster index of the 8x8 patch grid.
 *   R3  Ny = 0 fills 128.
 *   R4  BRL iff phi <= T_phi.
 *   R5  candidate windows lie inside the 48x48 support region; a candidate is valid iff
 *       every configured position (4 x positions + the Ny context positions) is
 *       available; candidate index = raster order of the window's top-left corner.
 *   R6  IDL rings: candidate patches at Chebyshev distance D from x0 belong to ring
 *       ceil(D / ring_step); after each ring nu = sum exp(-d/(2 sigma^2 Ny)) over all
 *       candidates so far (the sign of the exponent in Eq. (18) is read as negative,
 *       as Eq. (15) and the words "sum of raw weights" require); IDL iff nu >= T_nu;
 *       no ring reaching T_nu goes to HQL; no candidate at all falls back to BRL.
 *   R7  HQL: covariance with 1/M; ridge lambda = ridge_rel * tr(C_YY)/Ny + 1e-6 added
 *       to C_YY; beta grid 2^(k/2), k in [beta_kmin, beta_kmax]; beta* = the smallest
 *       grid value whose eps_y is within a relative beta_tie_rel of the minimum;
 *       I0 = the min(Ny+1, M-1) candidates with the smallest Mahalanobis distance to y0
 *       (ties to the lower index); leave-one-out predictions for i in I0; the alpha that
 *       minimises Eq. (11) in closed form, clamped to [0, 1] (0 if undefined).
 *   R8  every estimate is clipped to [0, 255] and written back unrounded (store_f32:
 *       rounded to binary32, to give a binary32 path under test identical inputs;
 *       quantize_inloop: rounded to the nearest integer, ties to even).
 *   R9  arbitrarily shaped loss (Sec. II: the method extends to any loss shape), given as
 *       a per-pixel mask: the unit of work stays the 16x16 block, and a block is worked on
 *       iff it holds a lost pixel; dependencies and R1 apply to those blocks.  Received
 *       pixels are available wherever they lie.  The patches to fill are the 2x2 patches
 *       of the block's grid holding a lost pixel.  x0 keeps the 2x2 shape of Fig. 1(a):
 *       its received pixels are not context (y0 never includes the patch itself, and the
 *       R2 count is over the 6x6 window less the patch), and only its lost pixels take
 *       the estimate.  With every pixel of a lost block lost this is the block method.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MB 16   /* block side (Sec. II) */
#define OR_REG 48  /* support region side: the lost block and its 8 neighbours */
#define OR_WIN 6   /* context window side (Sec. II) */
#define OR_NPOS (OR_REG - OR_WIN + 1) /* candidate window positions per axis: 43 */
#define OR_MAXCAND (OR_NPOS * OR_NPOS)

enum { OL_EMPTY = 0, OL_BRL = 1, OL_IDL = 2, OL_HQL = 3, OL_BRL_NOCAND = 4 };

typedef struct {
    double t_phi;        /* flatness threshold T_phi (Table I) */
    double t_nu;         /* normalisation threshold T_nu (Table I) */
    double sigma2;       /* IDL aperture sigma^2 (Sec. IV-B: 10) */
    int ring_step;       /* IDL ring width in pixels (R6) */
    double ridge_rel;    /* HQL ridge (R7) */
    int beta_kmin, beta_kmax; /* HQL beta grid (R7) */
    double beta_tie_rel; /* HQL beta tie tolerance (R7) */
    int concealed_is_support; /* R1 */
    int store_f32;       /* R8 variant: reconstructions are stored rounded to binary32 (the
                            storage precision of a path under test); arithmetic stays FP64 */
    int quantize_inloop; /* R8 variant: every estimate is written back into the support
                            rounded to an 8-bit integer (round half to even), as a decoder
                            that keeps 8-bit frames does; the trace keeps the estimate */
    double perturb;      /* sensitivity variant (test infrastructure, not the method): every
                            written-back estimate is moved by perturb * u before the clip of
                            R8, u in [-1, 1) drawn by SplitMix64 from (block, step, pixel,
                            perturb_seed); 0 leaves the method unchanged.  It measures how
                            far the sequential fill carries an error of a given size made
                            at one step, the way a path with that per-step error would */
    uint64_t perturb_seed;
} oracle_params;

typedef struct {
    int32_t mb;        /* raster index of the lost block */
    int32_t step;      /* fill step inside the block */
    int32_t patch;     /* patch index a*8+b inside the block */
    int32_t layer;     /* OL_* */
    int32_t ny;        /* context size */
    int32_t m;         /* number of candidates in the whole support (0 if not enumerated) */
    int32_t ring;      /* IDL: accepted ring (1-based); otherwise the number of rings tried */
    int32_t beta_idx;  /* HQL: index into the beta grid, else -1 */
    int32_t n0;        /* HQL: |I0| */
    int32_t pad;
    double phi;        /* flatness, Eq. (17) */
    double log_nu;     /* log of nu after the last ring evaluated, Eq. (18) */
    double alpha;      /* HQL alpha */
    double eps_best;   /* HQL eps_y(beta*) */
    double x[4];       /* the estimate after clipping */
    double margin_phi; /* |phi - T_phi| */
    double margin_nu;  /* min over evaluated rings of |log nu - log T_nu| */
    double margin_beta;/* min over grid values up to beta* of |eps/eps_min - (1+tie)| */
    double margin_i0;  /* relative gap between the n0-th and (n0+1)-th smallest distance */
    uint16_t i0[36];   /* I0 as candidate window indices wu*43+wv, ascending */
} oracle_trace_rec;

typedef struct {
    int64_t n_patches, n_empty, n_brl, n_idl, n_hql, n_brl_nocand;
    int64_t idl_ring_hist[16];
    int64_t idl_cand_evals;
    int64_t hql_cands;
} oracle_stats;

/* ------------------------------------------------------------------------------ */

typedef struct {
    const uint8_t* frame; int W, H, pitch;
    const uint8_t* mb_lost; int mbw, mbh;
    const uint8_t* px_lost; int px_pitch; /* R9: per-pixel loss, or NULL (whole blocks) */
    const oracle_params* p;
    double* out;               /* W*H values */
    int32_t* lost_index;       /* per block: raster rank among lost blocks, -1 received */
    oracle_trace_rec* trace;   /* n_lost*64 records or NULL */
    oracle_stats stats;        /* accumulated (merged after threads) */
} oracle_job;

typedef struct {
    /* per-thread scratch */
    double R[OR_REG][OR_REG];
    unsigned char A[OR_REG][OR_REG];
    int cand[OR_MAXCAND];      /* window top-left index wu*43+wv */
    double d[OR_MAXCAND];
    double *Z;                 /* M x (4+Ny) */
    double *V;                 /* M x Ny whitened contexts */
    oracle_stats st;
} oracle_scratch;

static int popcount_window(unsigned char A[OR_REG][OR_REG], int r0, int c0) {
    int n = 0;
    for (int r = 0; r < OR_WIN; r++)
        for (int c = 0; c < OR_WIN; c++) n += A[r0 + r][c0 + c] ? 1 : 0;
    return n;
}

static double clip255(double v) { return v < 0.0 ? 0.0 : (v > 255.0 ? 255.0 : v); }

/* SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number generators",
   OOPSLA 2014): the output function applied to a counter; 53 bits mapped to [-1, 1) */
uint64_t oracle_splitmix64(uint64_t x) {
    uint64_t z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static double splitmix_unit(uint64_t x) {
    return (double)(oracle_splitmix64(x) >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

/* is frame pixel (fy, fx) lost: its block's flag, or its own flag under R9 */
static int pixel_lost(const oracle_job* job, int fy, int fx) {
    if (job->px_lost) return job->px_lost[(size_t)fy * job->px_pitch + fx] != 0;
    return job->mb_lost[(fy / OR_MB) * job->mbw + fx / OR_MB] != 0;
}

/* is window position (r, c) of a 6x6 window one of the patch's own four positions */
static int in_patch(int r, int c) { return (r == 2 || r == 3) && (c == 2 || c == 3); }

/* Cholesky factorisation of an n x n SPD matrix (row-major, lda = n): A = L L^T. */
static int cholesky(double* a, int n) {
    for (int j = 0; j < n; j++) {
        double s = a[j * n + j];
        for (int k = 0; k < j; k++) s -= a[j * n + k] * a[j * n + k];
        if (!(s > 0.0)) return -1;
        double l = sqrt(s);
        a[j * n + j] = l;
        for (int i = j + 1; i < n; i++) {
            double t = a[i * n + j];
            for (int k = 0; k < j; k++) t -= a[i * n + k] * a[j * n + k];
            a[i * n + j] = t / l;
        }
        for (int i = 0; i < j; i++) a[i * n + j] = 0.0;
    }
    return 0;
}

/* Solve L v = b by forward substitution (L lower triangular, row-major). */
static void forward_solve(const double* L, int n, const double* b, double* v) {
    for (int i = 0; i < n; i++) {
        double s = b[i];
        for (int k = 0; k < i; k++) s -= L[i * n + k] * v[k];
        v[i] = s / L[i * n + i];
    }
}

/* Solve L^T v = b by back substitution. */
static void backward_solve_t(const double* L, int n, const double* b, double* v) {
    for (int i = n - 1; i >= 0; i--) {
        double s = b[i];
        for (int k = i + 1; k < n; k++) s -= L[k * n + i] * v[k];
        v[i] = s / L[i * n + i];
    }
}

/* HQL, Eq. (13): x0_hat = x0~(beta) + alpha C_XY C_YY^-1 (y0 - y0~(beta)).
 * z_j rows of Z are (x_j[4], y_j[Ny]); y0 has Ny entries. */
static void hql_estimate(oracle_scratch* s, const oracle_params* p, int M, int ny,
                         const double* y0, double xhat[4], oracle_trace_rec* tr) {
    const int nz = 4 + ny;
    double mu[36], C[36 * 36];
    /* sample mean and covariance of z_j, 1/M (Eq. (8), R7) */
    for (int k = 0; k < nz; k++) {
        double acc = 0.0;
        for (int j = 0; j < M; j++) acc += s->Z[j * nz + k];
        mu[k] = acc / M;
    }
    for (int a = 0; a < nz; a++)
        for (int b = 0; b < nz; b++) {
            double acc = 0.0;
            for (int j = 0; j < M; j++)
                acc += (s->Z[j * nz + a] - mu[a]) * (s->Z[j * nz + b] - mu[b]);
            C[a * nz + b] = acc / M;
        }
    /* C_YY with ridge (R7); C_XY */
    double Cyy[32 * 32], L[32 * 32], Cxy[4 * 32];
    double tr_yy = 0.0;
    for (int i = 0; i < ny; i++) tr_yy += C[(4 + i) * nz + 4 + i];
    double lambda = p->ridge_rel * tr_yy / ny + 1e-6;
    for (int i = 0; i < ny; i++)
        for (int k = 0; k < ny; k++)
            Cyy[i * ny + k] = C[(4 + i) * nz + 4 + k] + (i == k ? lambda : 0.0);
    for (int a = 0; a < 4; a++)
        for (int k = 0; k < ny; k++) Cxy[a * ny + k] = C[a * nz + 4 + k];
    memcpy(L, Cyy, sizeof(double) * ny * ny);
    if (cholesky(L, ny) != 0) {
        /* cannot happen for lambda > 0; keep the estimate defined */
        for (int a = 0; a < 4; a++) xhat[a] = mu[a];
        return;
    }
    /* Kmat = C_XY C_YY^-1, one row at a time: C_YY k_a = c_a (C_YY symmetric) */
    double Kmat[4 * 32];
    for (int a = 0; a < 4; a++) {
        double t[32];
        forward_solve(L, ny, &Cxy[a * ny], t);
        backward_solve_t(L, ny, t, &Kmat[a * ny]);
    }
    /* whitened contexts v_j = L^-1 y_j; Mahalanobis distance
       (y_i - y_j)^T C_YY^-1 (y_i - y_j) = ||v_i - v_j||^2 since L^-1 is linear */
    double v0[32];
    forward_solve(L, ny, y0, v0);
    for (int j = 0; j < M; j++) forward_solve(L, ny, &s->Z[j * nz + 4], &s->V[j * ny]);
    for (int j = 0; j < M; j++) {
        double acc = 0.0;
        for (int k = 0; k < ny; k++) {
            double e = v0[k] - s->V[j * ny + k];
            acc += e * e;
        }
        s->d[j] = acc;
    }
    double dmin = s->d[0];
    for (int j = 1; j < M; j++) if (s->d[j] < dmin) dmin = s->d[j];

    /* beta search, Eqs. (9)-(10): eps_y(beta) = ||y0 - sum_j w_j(beta) y_j||^2 with
       w_j from Eq. (6), H_YY = beta C_YY (exponent -d_j / (2 beta)) */
    const int nb = p->beta_kmax - p->beta_kmin + 1;
    double eps[64];
    for (int b = 0; b < nb; b++) {
        double beta = pow(2.0, 0.5 * (p->beta_kmin + b));
        double wsum = 0.0, yt[32];
        for (int k = 0; k < ny; k++) yt[k] = 0.0;
        for (int j = 0; j < M; j++) {
            double w = exp(-(s->d[j] - dmin) / (2.0 * beta));
            wsum += w;
            for (int k = 0; k < ny; k++) yt[k] += w * s->Z[j * nz + 4 + k];
        }
        double e = 0.0;
        for (int k = 0; k < ny; k++) {
            double r = y0[k] - yt[k] / wsum;
            e += r * r;
        }
        eps[b] = e;
    }
    double emin = eps[0];
    for (int b = 1; b < nb; b++) if (eps[b] < emin) emin = eps[b];
    int bstar = 0;
    for (int b = 0; b < nb; b++)
        if (eps[b] <= emin * (1.0 + p->beta_tie_rel)) { bstar = b; break; }
    /* distance of the decision to a flip: a grid value before beta* crossing into the
       tie band, or beta* itself (when it is not the minimiser) leaving it */
    double mb = INFINITY;
    for (int b = 0; b <= bstar; b++) {
        if (emin <= 0.0) break; /* exact zeros: no ambiguity */
        double r = eps[b] / emin;
        if (b == bstar && r == 1.0) continue;
        double g = fabs(r - (1.0 + p->beta_tie_rel));
        if (g < mb) mb = g;
    }
    const double beta_s = pow(2.0, 0.5 * (p->beta_kmin + bstar));

    /* x0~ and y0~ at beta*, Eqs. (4)-(5) */
    double xt0[4] = {0, 0, 0, 0}, yt0[32], wsum0 = 0.0;
    for (int k = 0; k < ny; k++) yt0[k] = 0.0;
    for (int j = 0; j < M; j++) {
        double w = exp(-(s->d[j] - dmin) / (2.0 * beta_s));
        wsum0 += w;
        for (int a = 0; a < 4; a++) xt0[a] += w * s->Z[j * nz + a];
        for (int k = 0; k < ny; k++) yt0[k] += w * s->Z[j * nz + 4 + k];
    }
    for (int a = 0; a < 4; a++) xt0[a] /= wsum0;
    for (int k = 0; k < ny; k++) yt0[k] /= wsum0;

    /* I0: the min(Ny+1, M-1) nearest candidates to y0 (Sec. III after Eq. (11)),
       ties to the lower candidate index: plain selection by repeated minimum */
    int n0 = ny + 1;
    if (n0 > M - 1) n0 = M - 1;
    if (n0 < 0) n0 = 0;
    int i0[36];
    unsigned char* taken = (unsigned char*)calloc((size_t)M, 1);
    for (int t = 0; t < n0; t++) {
        int best = -1;
        for (int j = 0; j < M; j++)
            if (!taken[j] && (best < 0 || s->d[j] < s->d[best])) best = j;
        taken[best] = 1;
        i0[t] = best;
    }
    double mi0 = INFINITY;
    if (n0 > 0 && n0 < M) {
        double dk = s->d[i0[n0 - 1]];
        int nxt = -1;
        for (int j = 0; j < M; j++)
            if (!taken[j] && (nxt < 0 || s->d[j] < s->d[nxt])) nxt = j;
        double gap = s->d[nxt] - dk;
        mi0 = dk > 0.0 ? gap / dk : (gap > 0.0 ? INFINITY : 0.0);
        if (gap == 0.0) mi0 = INFINITY; /* exact tie: resolved by index on both sides */
    }
    free(taken);

    /* alpha, Eqs. (11)-(12): x_i_hat(alpha) = x_i~ + alpha Kmat (y_i - y_i~) with
       leave-one-out predictions at beta*; eps_x is quadratic in alpha, so its
       minimiser is sum r_i.g_i / sum |g_i|^2 (R7) */
    double num = 0.0, den = 0.0;
    for (int t = 0; t < n0; t++) {
        const int i = i0[t];
        const double* vi = &s->V[i * ny];
        double dm = INFINITY;
        for (int j = 0; j < M; j++) {
            if (j == i) continue;
            double acc = 0.0;
            for (int k = 0; k < ny; k++) {
                double e = vi[k] - s->V[j * ny + k];
                acc += e * e;
            }
            s->d[j] = acc; /* d is no longer needed for y0 */
            if (acc < dm) dm = acc;
        }
        double xt[4] = {0, 0, 0, 0}, yt[32], ws = 0.0;
        for (int k = 0; k < ny; k++) yt[k] = 0.0;
        for (int j = 0; j < M; j++) {
            if (j == i) continue;
            double w = exp(-(s->d[j] - dm) / (2.0 * beta_s));
            ws += w;
            for (int a = 0; a < 4; a++) xt[a] += w * s->Z[j * nz + a];
            for (int k = 0; k < ny; k++) yt[k] += w * s->Z[j * nz + 4 + k];
        }
        double dy[32];
        for (int k = 0; k < ny; k++) dy[k] = s->Z[i * nz + 4 + k] - yt[k] / ws;
        for (int a = 0; a < 4; a++) {
            double g = 0.0;
            for (int k = 0; k < ny; k++) g += Kmat[a * ny + k] * dy[k];
            double r = s->Z[i * nz + a] - xt[a] / ws;
            num += r * g;
            den += g * g;
        }
    }
    double alpha = den > 0.0 ? num / den : 0.0;
    if (alpha < 0.0) alpha = 0.0;
    if (alpha > 1.0) alpha = 1.0;

    for (int a = 0; a < 4; a++) {
        double corr = 0.0;
        for (int k = 0; k < ny; k++) corr += Kmat[a * ny + k] * (y0[k] - yt0[k]);
        xhat[a] = xt0[a] + alpha * corr;
    }
    if (tr) {
        tr->beta_idx = bstar;
        tr->n0 = n0;
        tr->alpha = alpha;
        tr->eps_best = eps[bstar];
        tr->margin_beta = mb;
        tr->margin_i0 = mi0;
        /* I0 as window indices, ascending */
        int tmp[36];
        for (int t = 0; t < n0; t++) tmp[t] = s->cand[i0[t]];
        for (int a = 1; a < n0; a++) {
            int v = tmp[a], b = a - 1;
            while (b >= 0 && tmp[b] > v) { tmp[b + 1] = tmp[b]; b--; }
            tmp[b + 1] = v;
        }
        for (int t = 0; t < n0; t++) tr->i0[t] = (uint16_t)tmp[t];
    }
}

/* Conceal one lost block.  (by, bx) = block coordinates. */
static void conceal_block(oracle_job* job, oracle_scratch* s, int by, int bx) {
    const oracle_params* p = job->p;
    const int W = job->W, H = job->H;
    const int oy = by * OR_MB - OR_MB, ox = bx * OR_MB - OR_MB;
    const int my_rank = job->lost_index[by * job->mbw + bx];

    /* support region: the block and its 8 neighbours (Sec. II), availability per R1 */
    for (int r = 0; r < OR_REG; r++)
        for (int c = 0; c < OR_REG; c++) {
            int fy = oy + r, fx = ox + c;
            s->R[r][c] = 0.0;
            s->A[r][c] = 0;
            if (fy < 0 || fx < 0 || fy >= H || fx >= W) continue;
            int nb = (fy / OR_MB) * job->mbw + fx / OR_MB;
            int rank = job->lost_index[nb];
            if (rank < 0 || !pixel_lost(job, fy, fx)) { /* received (R9: wherever it lies) */
                s->R[r][c] = job->frame[(size_t)fy * job->pitch + fx];
                s->A[r][c] = 1;
            } else if (p->concealed_is_support && rank < my_rank) {
                s->R[r][c] = job->out[(size_t)fy * W + fx];
                s->A[r][c] = 1;
            }
        }

    /* patches of this block to fill: in the frame and holding a lost pixel (R9) */
    unsigned char filled[8][8], inframe[8][8];
    int npatch = 0;
    for (int a = 0; a < 8; a++)
        for (int b = 0; b < 8; b++) {
            filled[a][b] = 0;
            const int fy = by * OR_MB + 2 * a, fx = bx * OR_MB + 2 * b;
            inframe[a][b] = fy < H && fx < W &&
                            (pixel_lost(job, fy, fx) || pixel_lost(job, fy, fx + 1) ||
                             pixel_lost(job, fy + 1, fx) || pixel_lost(job, fy + 1, fx + 1));
            npatch += inframe[a][b];
        }

    for (int step = 0; step < npatch; step++) {
        /* R2: most available pixels in the 6x6 window less the patch (R9), ties to the
           lowest index */
        int pa = -1, pb = -1, best = -1;
        for (int a = 0; a < 8; a++)
            for (int b = 0; b < 8; b++) {
                if (!inframe[a][b] || filled[a][b]) continue;
                const int r0 = OR_MB + 2 * a, c0 = OR_MB + 2 * b;
                int n = popcount_window(s->A, r0 - 2, c0 - 2) - s->A[r0][c0] - s->A[r0][c0 + 1] -
                        s->A[r0 + 1][c0] - s->A[r0 + 1][c0 + 1];
                if (n > best) { best = n; pa = a; pb = b; }
            }
        const int pr = OR_MB + 2 * pa, pc = OR_MB + 2 * pb; /* patch top-left, region coords */
        const int wr = pr - 2, wc = pc - 2;                  /* window top-left */

        /* context y0: available pixels of the 6x6 window outside the patch, in window
           raster order (Sec. II, R9) */
        double y0[36];
        int yr[36], yc[36], ny = 0;
        for (int r = 0; r < OR_WIN; r++)
            for (int c = 0; c < OR_WIN; c++)
                if (!in_patch(r, c) && s->A[wr + r][wc + c]) {
                    y0[ny] = s->R[wr + r][wc + c];
                    yr[ny] = r;
                    yc[ny] = c;
                    ny++;
                }

        oracle_trace_rec* tr = NULL;
        if (job->trace) {
            tr = &job->trace[(size_t)my_rank * 64 + step];
            memset(tr, 0, sizeof(*tr));
            tr->mb = by * job->mbw + bx;
            tr->step = step;
            tr->patch = pa * 8 + pb;
            tr->ny = ny;
            tr->beta_idx = -1;
            tr->log_nu = -INFINITY;
            tr->margin_phi = INFINITY;
            tr->margin_nu = INFINITY;
            tr->margin_beta = INFINITY;
            tr->margin_i0 = INFINITY;
        }
        double xhat[4];
        int layer;
        s->st.n_patches++;
        if (ny == 0) {
            layer = OL_EMPTY; /* R3 */
            for (int a = 0; a < 4; a++) xhat[a] = 128.0;
            s->st.n_empty++;
        } else {
            double mx = y0[0], mn = y0[0], sum = 0.0;
            for (int k = 0; k < ny; k++) {
                if (y0[k] > mx) mx = y0[k];
                if (y0[k] < mn) mn = y0[k];
                sum += y0[k];
            }
            const double phi = mx - mn; /* Eq. (17) */
            if (tr) { tr->phi = phi; tr->margin_phi = fabs(phi - p->t_phi); }
            if (phi <= p->t_phi) {
                layer = OL_BRL; /* Eq. (16) */
                for (int a = 0; a < 4; a++) xhat[a] = sum / ny;
                s->st.n_brl++;
            } else {
                /* R5: candidates with the same spatial configuration */
                int M = 0;
                for (int wu = 0; wu < OR_NPOS; wu++)
                    for (int wv = 0; wv < OR_NPOS; wv++) {
                        int ok = s->A[wu + 2][wv + 2] && s->A[wu + 2][wv + 3] &&
                                 s->A[wu + 3][wv + 2] && s->A[wu + 3][wv + 3];
                        for (int k = 0; ok && k < ny; k++) ok = s->A[wu + yr[k]][wv + yc[k]];
                        if (ok) s->cand[M++] = wu * OR_NPOS + wv;
                    }
                if (tr) tr->m = M;
                if (M == 0) {
                    layer = OL_BRL_NOCAND; /* R6 */
                    for (int a = 0; a < 4; a++) xhat[a] = sum / ny;
                    s->st.n_brl_nocand++;
                } else {
                    /* IDL, Eq. (15) with the growing support of Sec. IV-B (R6) */
                    const double h = 2.0 * p->sigma2 * ny;
                    int maxring = 0;
                    int* ring = (int*)malloc(sizeof(int) * (size_t)M);
                    for (int j = 0; j < M; j++) {
                        int wu = s->cand[j] / OR_NPOS, wv = s->cand[j] % OR_NPOS;
                        int du = abs(wu + 2 - pr), dv = abs(wv + 2 - pc);
                        int D = du > dv ? du : dv;
                        ring[j] = (D + p->ring_step - 1) / p->ring_step;
                        if (ring[j] > maxring) maxring = ring[j];
                    }
                    double nu = 0.0, acc[4] = {0, 0, 0, 0};
                    int accepted = 0, k;
                    const double log_tnu = log(p->t_nu);
                    double mnu = INFINITY, lognu = -INFINITY;
                    for (k = 1; k <= maxring; k++) {
                        for (int j = 0; j < M; j++) {
                            if (ring[j] != k) continue;
                            const int wu = s->cand[j] / OR_NPOS, wv = s->cand[j] % OR_NPOS;
                            double d = 0.0;
                            for (int t = 0; t < ny; t++) {
                                double e = s->R[wu + yr[t]][wv + yc[t]] - y0[t];
                                d += e * e;
                            }
                            double rw = exp(-d / h);
                            nu += rw;
                            acc[0] += rw * s->R[wu + 2][wv + 2];
                            acc[1] += rw * s->R[wu + 2][wv + 3];
                            acc[2] += rw * s->R[wu + 3][wv + 2];
                            acc[3] += rw * s->R[wu + 3][wv + 3];
                            s->st.idl_cand_evals++;
                        }
                        lognu = log(nu);
                        double g = fabs(lognu - log_tnu);
                        if (g < mnu) mnu = g;
                        if (nu >= p->t_nu) { accepted = 1; break; }
                    }
                    free(ring);
                    if (tr) {
                        tr->log_nu = lognu;
                        tr->margin_nu = mnu;
                        tr->ring = accepted ? k : maxring;
                    }
                    if (accepted) {
                        layer = OL_IDL;
                        for (int a = 0; a < 4; a++) xhat[a] = acc[a] / nu;
                        s->st.n_idl++;
                        if (k < 16) s->st.idl_ring_hist[k]++;
                    } else {
                        layer = OL_HQL;
                        const int nz = 4 + ny;
                        for (int j = 0; j < M; j++) {
                            const int wu = s->cand[j] / OR_NPOS, wv = s->cand[j] % OR_NPOS;
                            double* z = &s->Z[j * nz];
                            z[0] = s->R[wu + 2][wv + 2];
                            z[1] = s->R[wu + 2][wv + 3];
                            z[2] = s->R[wu + 3][wv + 2];
                            z[3] = s->R[wu + 3][wv + 3];
                            for (int t = 0; t < ny; t++) z[4 + t] = s->R[wu + yr[t]][wv + yc[t]];
                        }
                        hql_estimate(s, p, M, ny, y0, xhat, tr);
                        s->st.n_hql++;
                        s->st.hql_cands += M;
                    }
                }
            }
        }
        /* R8: clip, write back into the support (end of Sec. III); R9: the lost pixels of
           the patch only (they are the unavailable ones) */
        const int fr[4] = {pr, pr, pr + 1, pr + 1}, fc[4] = {pc, pc + 1, pc, pc + 1};
        for (int a = 0; a < 4; a++) {
            if (p->perturb != 0.0) {
                const uint64_t key = (((uint64_t)(by * job->mbw + bx) * 64u + (uint64_t)step) * 4u +
                                      (uint64_t)a) ^ (p->perturb_seed * 0x100000001B3ull);
                xhat[a] += p->perturb * splitmix_unit(key);
            }
            xhat[a] = clip255(xhat[a]);
            if (p->store_f32) xhat[a] = (double)(float)xhat[a];
            if (s->A[fr[a]][fc[a]]) continue;
            s->R[fr[a]][fc[a]] = p->quantize_inloop ? nearbyint(xhat[a]) : xhat[a];
            s->A[fr[a]][fc[a]] = 1;
        }
        filled[pa][pb] = 1;
        if (tr) {
            tr->layer = layer;
            for (int a = 0; a < 4; a++) tr->x[a] = xhat[a];
        }
    }
    /* publish the block */
    for (int r = 0; r < OR_MB; r++)
        for (int c = 0; c < OR_MB; c++) {
            int fy = by * OR_MB + r, fx = bx * OR_MB + c;
            if (fy < H && fx < W) job->out[(size_t)fy * W + fx] = s->R[OR_MB + r][OR_MB + c];
        }
}

/* ------------------------------------------------------------------------------ */
/* scheduling: blocks of one dependency level are independent (R1) */

typedef struct {
    oracle_job* job;
    const int32_t* list;   /* block raster indices of this level */
    int n;
    volatile int next;
    pthread_mutex_t mu;
} level_work;

typedef struct { level_work* lw; oracle_scratch* s; } worker_arg;

static void* worker(void* argp) {
    worker_arg* wa = (worker_arg*)argp;
    level_work* lw = wa->lw;
    for (;;) {
        pthread_mutex_lock(&lw->mu);
        int i = lw->next++;
        pthread_mutex_unlock(&lw->mu);
        if (i >= lw->n) break;
        int b = lw->list[i];
        conceal_block(lw->job, wa->s, b / lw->job->mbw, b % lw->job->mbw);
    }
    return NULL;
}

static oracle_scratch* scratch_new(void) {
    oracle_scratch* s = (oracle_scratch*)calloc(1, sizeof(oracle_scratch));
    s->Z = (double*)malloc(sizeof(double) * OR_MAXCAND * 36);
    s->V = (double*)malloc(sizeof(double) * OR_MAXCAND * 32);
    return s;
}

static void scratch_free(oracle_scratch* s) {
    free(s->Z);
    free(s->V);
    free(s);
}

static int conceal_frame(const uint8_t* frame, int W, int H, int pitch, const uint8_t* mb_lost,
                         const uint8_t* px_lost, int px_pitch, const uint8_t* select,
                         const oracle_params* p, double* out, oracle_trace_rec* trace,
                         oracle_stats* stats, int nthreads) {
    const int mbw = (W + OR_MB - 1) / OR_MB, mbh = (H + OR_MB - 1) / OR_MB;
    oracle_job job;
    memset(&job, 0, sizeof(job));
    job.frame = frame; job.W = W; job.H = H; job.pitch = pitch;
    job.mb_lost = mb_lost; job.mbw = mbw; job.mbh = mbh; job.p = p;
    job.px_lost = px_lost; job.px_pitch = px_pitch;
    job.out = out; job.trace = trace;
    job.lost_index = (int32_t*)malloc(sizeof(int32_t) * (size_t)mbw * mbh);
    int nlost = 0;
    for (int b = 0; b < mbw * mbh; b++) job.lost_index[b] = mb_lost[b] ? nlost++ : -1;
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++)
            out[(size_t)y * W + x] = pixel_lost(&job, y, x) ? NAN : (double)frame[(size_t)y * pitch + x];
    /* which blocks to run: all lost, or the selected ones plus their ancestors */
    unsigned char* run = (unsigned char*)calloc((size_t)mbw * mbh, 1);
    for (int b = mbw * mbh - 1; b >= 0; b--) {
        if (!mb_lost[b]) continue;
        if (!select || select[b]) run[b] = 1;
        if (!run[b] || !p->concealed_is_support) continue;
        int by = b / mbw, bx = b % mbw;
        const int dy[4] = {-1, -1, -1, 0}, dx[4] = {-1, 0, 1, -1};
        for (int t = 0; t < 4; t++) {
            int ny = by + dy[t], nx = bx + dx[t];
            if (ny < 0 || nx < 0 || nx >= mbw) continue;
            if (mb_lost[ny * mbw + nx]) run[ny * mbw + nx] = 1;
        }
    }
    /* dependency levels: a lost block waits for its lost neighbours earlier in raster
       order (left, top-left, top, top-right) when those are support (R1) */
    int32_t* level = (int32_t*)malloc(sizeof(int32_t) * (size_t)mbw * mbh);
    int maxlevel = -1;
    for (int b = 0; b < mbw * mbh; b++) {
        level[b] = -1;
        if (!run[b]) continue;
        int lv = 0;
        if (p->concealed_is_support) {
            int by = b / mbw, bx = b % mbw;
            const int dy[4] = {-1, -1, -1, 0}, dx[4] = {-1, 0, 1, -1};
            for (int t = 0; t < 4; t++) {
                int ny = by + dy[t], nx = bx + dx[t];
                if (ny < 0 || nx < 0 || nx >= mbw) continue;
                int q = ny * mbw + nx;
                if (mb_lost[q] && level[q] + 1 > lv) lv = level[q] + 1;
            }
        }
        level[b] = lv;
        if (lv > maxlevel) maxlevel = lv;
    }
    if (nthreads < 1) nthreads = 1;
    oracle_scratch** sc = (oracle_scratch**)malloc(sizeof(void*) * (size_t)nthreads);
    for (int t = 0; t < nthreads; t++) sc[t] = scratch_new();
    int32_t* list = (int32_t*)malloc(sizeof(int32_t) * (size_t)mbw * mbh);
    for (int lv = 0; lv <= maxlevel; lv++) {
        int n = 0;
        for (int b = 0; b < mbw * mbh; b++) if (level[b] == lv) list[n++] = b;
        level_work lw;
        lw.job = &job; lw.list = list; lw.n = n; lw.next = 0;
        pthread_mutex_init(&lw.mu, NULL);
        int nt = nthreads < n ? nthreads : n;
        if (nt <= 1) {
            for (int i = 0; i < n; i++) conceal_block(&job, sc[0], list[i] / mbw, list[i] % mbw);
        } else {
            pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nt);
            worker_arg* wa = (worker_arg*)malloc(sizeof(worker_arg) * (size_t)nt);
            for (int t = 0; t < nt; t++) {
                wa[t].lw = &lw;
                wa[t].s = sc[t];
                pthread_create(&th[t], NULL, worker, &wa[t]);
            }
            for (int t = 0; t < nt; t++) pthread_join(th[t], NULL);
            free(th);
            free(wa);
        }
        pthread_mutex_destroy(&lw.mu);
    }
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        for (int t = 0; t < nthreads; t++) {
            oracle_stats* a = &sc[t]->st;
            stats->n_patches += a->n_patches; stats->n_empty += a->n_empty;
            stats->n_brl += a->n_brl; stats->n_idl += a->n_idl; stats->n_hql += a->n_hql;
            stats->n_brl_nocand += a->n_brl_nocand;
            for (int k = 0; k < 16; k++) stats->idl_ring_hist[k] += a->idl_ring_hist[k];
            stats->idl_cand_evals += a->idl_cand_evals;
            stats->hql_cands += a->hql_cands;
        }
    }
    for (int t = 0; t < nthreads; t++) scratch_free(sc[t]);
    free(sc);
    free(list);
    free(level);
    free(run);
    free(job.lost_index);
    return 0;
}

static int bad_args(int W, int H, int pitch, const oracle_params* p) {
    if (W <= 0 || H <= 0 || (W & 1) || (H & 1) || pitch < W || p->ring_step < 1) return 1;
    if (p->beta_kmax < p->beta_kmin || p->beta_kmax - p->beta_kmin >= 64) return 1;
    return 0;
}

/*
 * Conceal every lost block of one frame.
 *   frame: H rows of `pitch` bytes; mb_lost: ceil(H/16) x ceil(W/16) flags (1 = lost).
 *   select: NULL, or per-block flags restricting the work to the selected lost blocks
 *           and the lost blocks they depend on (for sampled checks of large frames).
 *   out: W*H doubles; received pixels are copied, lost pixels of skipped blocks are NaN.
 *   trace: NULL or n_lost*64 records, indexed by raster rank among lost blocks.
 * Returns 0, or -1 on bad arguments (odd sizes).
 */
int oracle_conceal(const uint8_t* frame, int W, int H, int pitch, const uint8_t* mb_lost,
                   const uint8_t* select, const oracle_params* p, double* out,
                   oracle_trace_rec* trace, oracle_stats* stats, int nthreads) {
    if (bad_args(W, H, pitch, p)) return -1;
    return conceal_frame(frame, W, H, pitch, mb_lost, NULL, 0, select, p, out, trace, stats,
                         nthreads);
}

/*
 * The same for an arbitrarily shaped loss (R9).
 *   px_lost: H rows of `px_pitch` flags (1 = lost).  The blocks worked on are those holding
 *   a lost pixel; select, trace and the record index refer to those blocks.
 */
int oracle_conceal_px(const uint8_t* frame, int W, int H, int pitch, const uint8_t* px_lost,
                      int px_pitch, const uint8_t* select, const oracle_params* p, double* out,
                      oracle_trace_rec* trace, oracle_stats* stats, int nthreads) {
    if (bad_args(W, H, pitch, p) || px_pitch < W) return -1;
    const int mbw = (W + OR_MB - 1) / OR_MB, mbh = (H + OR_MB - 1) / OR_MB;
    uint8_t* mb_lost = (uint8_t*)calloc((size_t)mbw * mbh, 1);
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++)
            if (px_lost[(size_t)y * px_pitch + x]) mb_lost[(y / OR_MB) * mbw + x / OR_MB] = 1;
    int rc = conceal_frame(frame, W, H, pitch, mb_lost, px_lost, px_pitch, select, p, out, trace,
                           stats, nthreads);
    free(mb_lost);
    return rc;
}

int oracle_trace_rec_size(void) { return (int)sizeof(oracle_trace_rec); }
int oracle_params_size(void) { return (int)sizeof(oracle_params); }
int oracle_stats_size(void) { return (int)sizeof(oracle_stats); }

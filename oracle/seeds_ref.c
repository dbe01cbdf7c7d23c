/*
 * seeds_ref.c -- the oracle for the SEEDS hot path: a plain, slow,
 * single-threaded CPU statement of what the GPU library computes.
 *
 * TEST INFRASTRUCTURE ONLY.  The test suite, the package smoke check and the
 * benchmark's CPU-baseline / reference leg are the only callers.  Nothing in
 * this file is shared with the CUDA path (no header, helper, table or
 * generator), and the CUDA path never loads it.
 *
 * Method: M. Van den Bergh, X. Boix, G. Roig, L. Van Gool, "SEEDS:
 * Superpixels Extracted via Energy-Driven Sampling" (arXiv 1309.3848).
 *
 *   partition s : {1..N} -> {1..K}, sets A_k ........... Sec. 3, Eqs. 1-2
 *   colour histogram c_A(j) ............................ Sec. 4.1, Eq. 4
 *   label-patch histogram b_{N_i}(k), G(s) ............. Sec. 4.2, Eqs. 6-7
 *   grid initialisation, block hierarchy ............... Sec. 5.1
 *   block / pixel proposals ............................ Sec. 5.2
 *   intersection test (Prop. 1) ........................ Sec. 5.3, App. A.1
 *   single-lookup pixel test ........................... Sec. 5.3 (Fig. 6)
 *   label-patch test (Prop. 2) ......................... Sec. 5.3, App. A.2
 *   incremental histogram update ....................... Sec. 5.3 (last part)
 *
 * Readings taken where the paper is silent or loose (R-numbers; the same
 * list, with reasons, is kept in the repository's design notes):
 *   R1  colour bins from the raw RGB bytes: channel value v falls in bin
 *       b = floor(v*B/256); bin index j = bR*B*B + bG*B + bB.
 *   R2  colour histograms are normalised by |A| (App. A.1); label-patch
 *       histograms by the constant Z = 9, also for patches clipped at the
 *       image border, which keeps Prop. 2 exact.
 *   R3  grid: gx = max(1, round(sqrt(K*W/H))), gy = max(1, round(K/gx))
 *       (round half away from zero), K_actual = gx*gy; superpixel column
 *       edges floor(i*W/gx); level-l block column edges
 *       floor(i*W/(gx*2^(L-l+1))), rows likewise.  Level L blocks are a
 *       quarter superpixel (2x2 per superpixel), each finer level splits a
 *       block 2x2; the grids nest exactly.  Needs gx*2^L <= W, gy*2^L <= H.
 *   R4  L block levels (L = largest) then one pixel level; every level
 *       runs iters_per_level iterations.
 *   R5  a unit (block or pixel) is a boundary unit when a 4-neighbour unit
 *       of the same level has another label; its candidates are the
 *       distinct other labels among its 4-neighbours; the best candidate is
 *       the argmax of the score, ties to the smallest label id.
 *   R6  schedule: each iteration has four phases (py,px) = (0,0),(0,1),
 *       (1,0),(1,1); phase units are those with bx%2==px and by%2==py.
 *       All decisions of a phase read the labels and histograms as they
 *       were when the phase began; all accepted moves are applied after.
 *   R7  validity: superpixels are 4-connected.  Unit u may leave k only if
 *       (i) some 4-neighbour of u has label k and (ii) all k-labelled
 *       4-neighbours lie in one 4-connected run of k-labelled cells of u's
 *       8-ring (cells outside the grid are not k).
 *   R8  a move is accepted only if the score strictly increases.
 *   R9  every normalised comparison is an exact cross-multiplication
 *       (here in 128-bit integers).
 *   R10 pixel score: f(n) = D*c_An(j) + gamma*(G_n + |K_p|),
 *       f_stay = D*c_{Ak\p}(j) + gamma*G_k, D = N^4 = 81, where
 *       G_x = sum_{i in K_p} b_{N_i}(x) in counts (Prop. 2); blocks use the
 *       intersection alone (no G, Sec. 5.3).
 *   R11 (tests only) the paper's Prop. 1 agreement figures (Sec. 5.3,
 *       6.2) are two different poolings; they serve as a loose band.
 *   R12 s_t, described in Sec. 5 as the partition of lowest energy found,
 *       is the highest: the method maximises the energy.
 *   R13 K_p and N_i contain in-image pixels only.
 *   R16 colour space LAB (Sec. 6.2), optional: the bins of R1 taken over
 *       the 8-bit CIE L*a*b* code of each pixel (sRGB, D65; L* scaled by
 *       255/100, a* and b* offset by 128), computed in exact integer fixed
 *       point from two small tables of the published curves (see
 *       rgb_to_lab8).
 *   R15 anytime termination (Sec. 5.4): stopping after the first n ops of
 *       the schedule (init; per block level its phases and a descent; the
 *       pixel phases; the output) yields the partition as it stands, each
 *       pixel labelled by its unit at the current level.
 *   R17 means-based pixel updates (SPM, Sec. 6.3, run as the last pixel
 *       iterations, Sec. 6.5), optional: means_iters more pixel iterations
 *       of four parity phases in which a boundary pixel that may leave
 *       (R5, R7) moves to the candidate whose mean is nearest in SLIC's
 *       distance, colour codes plus (m/S)^2 times the squared distance to
 *       the superpixel's centroid (S^2 = N/K, m = compactness), if strictly
 *       nearer than its own superpixel's mean taken with the pixel in it;
 *       means from the phase-start state; no boundary term; evaluated in
 *       IEEE single precision in the order written in means_distance (a
 *       mean is its sum times the reciprocal of the size), so that any
 *       implementation doing the same operations decides the same way.
 *   R18 edge snapping (the edge prior of Sec. 6.4), optional: a boundary
 *       between 4-neighbour pixels lies on a colour edge when the L1
 *       distance of their colour codes (R1 bytes or R16 codes) is at least
 *       edge_threshold; a pixel with a 4-neighbour of another label across
 *       such an edge is snapped and no longer moves (pixel phases and R17
 *       means phases; blocks are not affected).
 *   R19 compactness prior (the second boundary prior of Sec. 6.4),
 *       optional: in the histogram pixel phases the score of every option
 *       loses w*D*d^2/S^2, where d^2 is the squared distance of the pixel to
 *       the option's centre of gravity (the stay option's with the pixel in
 *       it, as in R17), S^2 = N/K the nominal superpixel area, D = 81 and
 *       w = compact_prior/16.  The paper gives no formula, and the exact
 *       rational compare would overflow 128 bits, so with the prior on the
 *       whole pixel score is evaluated in IEEE single precision in the order
 *       written in compact_score (the colour term by one division, the
 *       centroid as its sum times the reciprocal of the size), centres from
 *       the phase-start state; blocks are not affected.  With
 *       compact_prior = 0 the exact integer test of R10 applies.
 *   R20 SPM on its own (Sec. 6.3): iters_per_level = 0 with means_iters > 0
 *       runs no histogram iteration: the block levels only descend, and the
 *       means-based iterations start from the grid.
 *   R14 sequential mode (quality reference only): per iteration the units
 *       are visited in a random permutation (SplitMix64 + Fisher-Yates),
 *       each boundary unit proposes one uniformly drawn candidate, and an
 *       accepted move is applied at once.  The generator, the visiting
 *       order and the candidate pick are pinned (published SplitMix64
 *       outputs; uniformity over all orders and over the candidates).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define REF_MAX_LEVELS 15

typedef __int128 i128;

typedef struct {
    int32_t width, height;
    int32_t num_superpixels;
    int32_t block_levels;
    int32_t bins_per_channel;
    int32_t iters_per_level;
    int32_t patch;      /* 0 = no boundary term, 3 = 3x3 patches */
    int32_t gamma_num;
    int32_t gamma_den;
    int32_t color_space; /* 0 = RGB bytes (R1), 1 = CIE L*a*b* (R16) */
    int32_t means_iters; /* R17: means-based pixel iterations after the histogram ones */
    int32_t compactness; /* R17: SLIC's m, weight of the spatial distance */
    int32_t edge_threshold; /* R18: colour-edge strength that snaps a pixel boundary (0 = off) */
    int32_t compact_prior;  /* R19: weight of the compactness prior, in 1/16 (0 = off) */
} ref_params;

typedef struct {
    ref_params p;
    int W, H, L, B, nbins;
    int gx, gy, K;
    /* unit grids: level 0 = pixels, level l >= 1 = blocks */
    int nbx[REF_MAX_LEVELS + 1], nby[REF_MAX_LEVELS + 1];
    int *xe[REF_MAX_LEVELS + 1], *ye[REF_MAX_LEVELS + 1];
    int *bin;        /* colour bin of every pixel */
    int *lab;        /* s(i) for every pixel */
    int64_t *hist;   /* K x nbins: |A_k| * c_{A_k}(j) */
    int64_t *size;   /* |A_k| */
    int64_t *tmp_l;  /* dense histogram of the unit being evaluated */
    int64_t *tmp_a;  /* A_k \ L */
    int32_t *moves;  /* (unit, k, n) triples of the current phase */
    int64_t moves_cap;
    uint8_t *code;         /* colour code (the channels the bins are taken from) of every pixel */
    int64_t *msum;         /* R17: per superpixel: sums of the 3 codes, of x and of y */
    float means_w;         /* R17: m^2 K / N, the spatial weight (m/S)^2 with S^2 = N/K */
    float compact_w;       /* R19: (compact_prior/16) * D * K / N, the weight of d^2 */
    float gamma_f;         /* R19: gamma as a float (0 without patches) */
    int64_t lab_lin[256];  /* R16: sRGB byte -> linear light * 2^24 */
    int64_t lab_m[3][3];   /* R16: linear RGB -> XYZ / white, * 2^20 */
} ref_state;

enum { REF_OK = 0, REF_EINVAL = -1, REF_EGEOM = -2, REF_ENOMEM = -4, REF_ESIZE = -7 };

/* ------------------------------------------------------------------ */
/* geometry (R3)                                                        */
/* ------------------------------------------------------------------ */

static int64_t edge_at(int64_t i, int64_t extent, int64_t count)
{
    return (i * extent) / count; /* floor for non-negative operands */
}

int ref_check_params(const ref_params *p)
{
    if (!p) return REF_EINVAL;
    if (p->width < 1 || p->height < 1 || p->width > 32768 || p->height > 32768) return REF_EINVAL;
    if ((int64_t)p->width * p->height > 0x7fffffffLL) return REF_EINVAL;
    if (p->num_superpixels < 1) return REF_EINVAL;
    if (p->block_levels < 0 || p->block_levels > REF_MAX_LEVELS) return REF_EINVAL;
    if (p->bins_per_channel < 1 || p->bins_per_channel > 16) return REF_EINVAL;
    /* R20: no histogram iteration only for a means-only run (SPM) */
    if (p->iters_per_level < 0 || p->iters_per_level > 1000) return REF_EINVAL;
    if (p->iters_per_level == 0 && p->means_iters == 0) return REF_EINVAL;
    if (p->patch != 0 && p->patch != 3) return REF_EINVAL;
    if (p->gamma_num < 0 || p->gamma_num > 1024) return REF_EINVAL;
    if (p->gamma_den < 1 || p->gamma_den > 1024) return REF_EINVAL;
    if (p->color_space != 0 && p->color_space != 1) return REF_EINVAL;
    if (p->means_iters < 0 || p->means_iters > 1000) return REF_EINVAL;
    if (p->compactness < 0 || p->compactness > 1024) return REF_EINVAL;
    if (p->edge_threshold < 0 || p->edge_threshold > 765) return REF_EINVAL;
    if (p->compact_prior < 0 || p->compact_prior > 1024) return REF_EINVAL;
    return REF_OK;
}

/* R3: superpixel grid gx x gy from the requested count. */
int ref_grid(const ref_params *p, int32_t *gx_out, int32_t *gy_out)
{
    int rc = ref_check_params(p);
    if (rc) return rc;
    double K = p->num_superpixels, W = p->width, H = p->height;
    long gx = lround(sqrt(K * W / H));
    if (gx < 1) gx = 1;
    long gy = lround(K / (double)gx);
    if (gy < 1) gy = 1;
    if (gx * gy > 65535) return REF_EINVAL;
    *gx_out = (int32_t)gx;
    *gy_out = (int32_t)gy;
    if ((gx << p->block_levels) > p->width || (gy << p->block_levels) > p->height) return REF_EGEOM;
    return REF_OK;
}

void ref_destroy(ref_state *st)
{
    if (!st) return;
    for (int l = 0; l <= REF_MAX_LEVELS; ++l) {
        free(st->xe[l]);
        free(st->ye[l]);
    }
    free(st->bin);
    free(st->lab);
    free(st->hist);
    free(st->size);
    free(st->tmp_l);
    free(st->tmp_a);
    free(st->moves);
    free(st->code);
    free(st->msum);
    free(st);
}

static void lab_tables(ref_state *st);

int ref_create(const ref_params *p, ref_state **out)
{
    int32_t gx, gy;
    int rc = ref_grid(p, &gx, &gy);
    if (rc) return rc;
    ref_state *st = (ref_state *)calloc(1, sizeof(ref_state));
    if (!st) return REF_ENOMEM;
    st->p = *p;
    st->W = p->width;
    st->H = p->height;
    st->L = p->block_levels;
    st->B = p->bins_per_channel;
    st->nbins = st->B * st->B * st->B;
    st->gx = gx;
    st->gy = gy;
    st->K = gx * gy;
    int64_t N = (int64_t)st->W * st->H;

    /* level 0: every pixel is its own unit */
    st->nbx[0] = st->W;
    st->nby[0] = st->H;
    for (int l = 1; l <= st->L; ++l) {
        st->nbx[l] = gx << (st->L - l + 1);
        st->nby[l] = gy << (st->L - l + 1);
    }
    for (int l = 0; l <= st->L; ++l) {
        st->xe[l] = (int *)malloc(sizeof(int) * (st->nbx[l] + 1));
        st->ye[l] = (int *)malloc(sizeof(int) * (st->nby[l] + 1));
        if (!st->xe[l] || !st->ye[l]) { ref_destroy(st); return REF_ENOMEM; }
        for (int i = 0; i <= st->nbx[l]; ++i) st->xe[l][i] = (int)edge_at(i, st->W, st->nbx[l]);
        for (int i = 0; i <= st->nby[l]; ++i) st->ye[l][i] = (int)edge_at(i, st->H, st->nby[l]);
    }
    st->code = (uint8_t *)calloc((size_t)N * 3, 1);
    st->msum = (int64_t *)calloc((size_t)st->K * 5, sizeof(int64_t));
    st->means_w = (float)((int64_t)p->compactness * p->compactness * st->K) / (float)N;
    st->compact_w = (float)((int64_t)p->compact_prior * 81 * st->K) / (float)((int64_t)16 * N);
    st->gamma_f = p->patch == 3 ? (float)p->gamma_num / (float)p->gamma_den : 0.0f;
    st->bin = (int *)calloc((size_t)N, sizeof(int));
    st->lab = (int *)calloc((size_t)N, sizeof(int));
    st->hist = (int64_t *)calloc((size_t)st->K * st->nbins, sizeof(int64_t));
    st->size = (int64_t *)calloc((size_t)st->K, sizeof(int64_t));
    st->tmp_l = (int64_t *)calloc((size_t)st->nbins, sizeof(int64_t));
    st->tmp_a = (int64_t *)calloc((size_t)st->nbins, sizeof(int64_t));
    /* a phase holds at most ceil(nbx/2)*ceil(nby/2) units; level 0 is the largest grid */
    st->moves_cap = (int64_t)((st->W + 1) / 2) * ((st->H + 1) / 2);
    st->moves = (int32_t *)malloc(sizeof(int32_t) * 3 * st->moves_cap);
    if (!st->bin || !st->lab || !st->hist || !st->size || !st->tmp_l || !st->tmp_a || !st->moves || !st->code ||
        !st->msum) {
        ref_destroy(st);
        return REF_ENOMEM;
    }
    lab_tables(st);
    *out = st;
    return REF_OK;
}

int ref_info(const ref_state *st, int32_t *gx, int32_t *gy, int32_t *K, int32_t *nbins)
{
    *gx = st->gx;
    *gy = st->gy;
    *K = st->K;
    *nbins = st->nbins;
    return REF_OK;
}

/* unit grid and edges of one level (level 0 = pixels) */
int ref_level_grid(const ref_state *st, int level, int32_t *nbx, int32_t *nby, int32_t *xe, int32_t *ye)
{
    if (level < 0 || level > st->L) return REF_EINVAL;
    *nbx = st->nbx[level];
    *nby = st->nby[level];
    if (xe) for (int i = 0; i <= st->nbx[level]; ++i) xe[i] = st->xe[level][i];
    if (ye) for (int i = 0; i <= st->nby[level]; ++i) ye[i] = st->ye[level][i];
    return REF_OK;
}

/* ------------------------------------------------------------------ */
/* colour bins (R1), initial grid (Sec. 5.1) and histograms (Eq. 4)      */
/* ------------------------------------------------------------------ */

static int channel_bin(int v, int B)
{
    /* the bin whose interval [b*256/B, (b+1)*256/B) holds v */
    for (int b = 0; b < B; ++b)
        if (v * B >= b * 256 && v * B < (b + 1) * 256) return b;
    return B - 1; /* unreachable for 0 <= v <= 255 */
}

/* R16: CIE 1976 L*a*b* of sRGB under D65 (Sec. 6.2 reports LAB as the
 * best colour space), in exact integer fixed point.  Two tables come from
 * the published definitions in double precision, rounded to integers: the
 * sRGB decoding curve (IEC 61966-2-1) as linear light * 2^24, and the sRGB
 * to XYZ matrix with each row divided by its sum (the D65 white) * 2^20.
 * The rest is integer arithmetic: t = T / 2^44 per channel, f(t) * 2^20
 * (floor), and the 8-bit code of each coordinate -- L* * 255/100, a* + 128,
 * b* + 128, each rounded half up and clamped to [0, 255]. */
static const double SRGB_TO_XYZ[3][3] = {
    {0.4124, 0.3576, 0.1805}, {0.2126, 0.7152, 0.0722}, {0.0193, 0.1192, 0.9505}};

static double srgb_decode(int v)
{
    double c = v / 255.0;
    return c <= 0.04045 ? c / 12.92 : pow((c + 0.055) / 1.055, 2.4);
}

static void lab_tables(ref_state *st)
{
    for (int v = 0; v < 256; ++v) st->lab_lin[v] = llround(srgb_decode(v) * 16777216.0);
    for (int i = 0; i < 3; ++i) {
        double white = SRGB_TO_XYZ[i][0] + SRGB_TO_XYZ[i][1] + SRGB_TO_XYZ[i][2];
        for (int j = 0; j < 3; ++j) st->lab_m[i][j] = llround(SRGB_TO_XYZ[i][j] / white * 1048576.0);
    }
}

/* floor(cbrt(n)) for 0 <= n < 2^60.2, by bisection */
static int64_t icbrt_floor(int64_t n)
{
    int64_t lo = 0, hi = ((int64_t)1 << 20) + ((int64_t)1 << 16);
    while (lo < hi) {
        int64_t mid = (lo + hi + 1) / 2;
        if (mid * mid * mid <= n)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

/* floor(f(t) * 2^20) for t = T / 2^44, where f(t) = t^(1/3) above
 * (6/29)^3 = 216/24389 and the line t / (3 (6/29)^2) + 4/29 =
 * (24389 t + 432) / 3132 below */
static int64_t lab_f_q20(int64_t T)
{
    if (T * 24389 > ((int64_t)216 << 44)) return icbrt_floor(T << 16); /* cbrt(t * 2^60) */
    return (24389 * T + ((int64_t)432 << 44)) / ((int64_t)3132 << 24);
}

static int64_t floor_div(int64_t a, int64_t b)
{
    int64_t q = a / b;
    return (a % b != 0 && ((a < 0) != (b < 0))) ? q - 1 : q;
}

static int clamp_byte(int64_t v) { return v < 0 ? 0 : v > 255 ? 255 : (int)v; }

static void rgb_to_lab8(const ref_state *st, int r, int g, int b, int out[3])
{
    int64_t f[3];
    for (int i = 0; i < 3; ++i) {
        int64_t T = st->lab_m[i][0] * st->lab_lin[r] + st->lab_m[i][1] * st->lab_lin[g] +
                    st->lab_m[i][2] * st->lab_lin[b];
        f[i] = lab_f_q20(T);
    }
    int64_t Lq = 116 * f[1] - ((int64_t)16 << 20); /* L* * 2^20 */
    out[0] = clamp_byte(floor_div(Lq * 255 + ((int64_t)50 << 20), (int64_t)100 << 20));
    out[1] = clamp_byte(floor_div(500 * (f[0] - f[1]) + ((int64_t)128 << 20) + (1 << 19), (int64_t)1 << 20));
    out[2] = clamp_byte(floor_div(200 * (f[1] - f[2]) + ((int64_t)128 << 20) + (1 << 19), (int64_t)1 << 20));
}

/* the 8-bit L*a*b* codes of n RGB triples (test hook) */
void ref_lab8(const ref_state *st, const uint8_t *rgb, int64_t n, uint8_t *out)
{
    for (int64_t i = 0; i < n; ++i) {
        int c[3];
        rgb_to_lab8(st, rgb[3 * i], rgb[3 * i + 1], rgb[3 * i + 2], c);
        for (int q = 0; q < 3; ++q) out[3 * i + q] = (uint8_t)c[q];
    }
}

/* index of the interval [e[i], e[i+1]) that holds v */
static int find_interval(const int *e, int n, int v)
{
    for (int i = 0; i < n; ++i)
        if (v >= e[i] && v < e[i + 1]) return i;
    return -1;
}

/* recount c_{A_k} (unnormalised) and |A_k| from the labels */
static void recount_histograms(ref_state *st)
{
    int64_t N = (int64_t)st->W * st->H;
    memset(st->hist, 0, sizeof(int64_t) * (size_t)st->K * st->nbins);
    memset(st->size, 0, sizeof(int64_t) * (size_t)st->K);
    for (int64_t i = 0; i < N; ++i) {
        st->hist[(int64_t)st->lab[i] * st->nbins + st->bin[i]] += 1;
        st->size[st->lab[i]] += 1;
    }
}

int ref_init(ref_state *st, const uint8_t *rgb, int64_t row_stride)
{
    if (!rgb || row_stride < 3 * (int64_t)st->W) return REF_EINVAL;
    int B = st->B;
    /* superpixel edges (the level-L blocks joined 2x2) */
    int *sxe = (int *)malloc(sizeof(int) * (st->gx + 1));
    int *sye = (int *)malloc(sizeof(int) * (st->gy + 1));
    if (!sxe || !sye) { free(sxe); free(sye); return REF_ENOMEM; }
    for (int i = 0; i <= st->gx; ++i) sxe[i] = (int)edge_at(i, st->W, st->gx);
    for (int i = 0; i <= st->gy; ++i) sye[i] = (int)edge_at(i, st->H, st->gy);
    for (int y = 0; y < st->H; ++y) {
        int sy = find_interval(sye, st->gy, y);
        for (int x = 0; x < st->W; ++x) {
            const uint8_t *px = rgb + (int64_t)y * row_stride + 3 * (int64_t)x;
            int c[3] = {px[0], px[1], px[2]};
            if (st->p.color_space == 1) rgb_to_lab8(st, px[0], px[1], px[2], c);
            for (int q = 0; q < 3; ++q) st->code[3 * ((int64_t)y * st->W + x) + q] = (uint8_t)c[q];
            int br = channel_bin(c[0], B), bg = channel_bin(c[1], B), bb = channel_bin(c[2], B);
            int sx = find_interval(sxe, st->gx, x);
            st->bin[(int64_t)y * st->W + x] = br * B * B + bg * B + bb;
            st->lab[(int64_t)y * st->W + x] = sy * st->gx + sx;
        }
    }
    free(sxe);
    free(sye);
    recount_histograms(st);
    return REF_OK;
}

/* ------------------------------------------------------------------ */
/* unit helpers                                                         */
/* ------------------------------------------------------------------ */

/* label of unit (bx,by) at a level: the label of its first pixel; units
 * are label-homogeneous (blocks move whole, levels run coarse to fine) */
static int unit_label(const ref_state *st, int level, int bx, int by)
{
    if (bx < 0 || by < 0 || bx >= st->nbx[level] || by >= st->nby[level]) return -1;
    int x = st->xe[level][bx], y = st->ye[level][by];
    return st->lab[(int64_t)y * st->W + x];
}

/* R7: local validity test on the 8-ring of unit (bx,by) for leaving label k.
 * Ring order walks around the unit; odd positions are the 4-neighbours, and
 * consecutive positions are 4-adjacent, so connected sets of ring cells are
 * runs of consecutive positions. */
static const int RING_DX[8] = {-1, 0, 1, 1, 1, 0, -1, -1};
static const int RING_DY[8] = {-1, -1, -1, 0, 1, 1, 1, 0};

static int leaving_keeps_connected(const ref_state *st, int level, int bx, int by, int k)
{
    int isk[8];
    int nk4 = 0, nk = 0;
    for (int r = 0; r < 8; ++r) {
        isk[r] = unit_label(st, level, bx + RING_DX[r], by + RING_DY[r]) == k;
        nk += isk[r];
        if (r & 1) nk4 += isk[r];
    }
    if (nk4 == 0) return 0;        /* (i) no k-labelled 4-neighbour */
    if (nk == 8) return 1;         /* whole ring is k: one run */
    int start = 0;
    while (isk[start]) ++start;    /* a position outside every run */
    int runs_with_4 = 0, in_run = 0, run_has_4 = 0;
    for (int t = 1; t <= 8; ++t) {
        int r = (start + t) % 8;
        if (isk[r]) {
            if (!in_run) { in_run = 1; run_has_4 = 0; }
            if (r & 1) run_has_4 = 1;
        } else if (in_run) {
            in_run = 0;
            runs_with_4 += run_has_4;
        }
    }
    /* the walk ends on `start`, which is not k, so every run was closed */
    return runs_with_4 == 1;
}

/* R5: distinct labels != k among the 4-neighbours, ascending */
static int candidates(const ref_state *st, int level, int bx, int by, int k, int cand[4])
{
    static const int DX[4] = {-1, 1, 0, 0}, DY[4] = {0, 0, -1, 1};
    int nc = 0;
    for (int d = 0; d < 4; ++d) {
        int n = unit_label(st, level, bx + DX[d], by + DY[d]);
        if (n < 0 || n == k) continue;
        int seen = 0;
        for (int c = 0; c < nc; ++c) seen |= cand[c] == n;
        if (!seen) cand[nc++] = n;
    }
    for (int a = 1; a < nc; ++a) /* insertion sort */
        for (int b = a; b > 0 && cand[b - 1] > cand[b]; --b) {
            int t = cand[b]; cand[b] = cand[b - 1]; cand[b - 1] = t;
        }
    return nc;
}

/* dense colour histogram of the pixels of unit (bx,by); returns |L| */
static int64_t unit_histogram(const ref_state *st, int level, int bx, int by, int64_t *h)
{
    memset(h, 0, sizeof(int64_t) * st->nbins);
    int64_t m = 0;
    for (int y = st->ye[level][by]; y < st->ye[level][by + 1]; ++y)
        for (int x = st->xe[level][bx]; x < st->xe[level][bx + 1]; ++x) {
            h[st->bin[(int64_t)y * st->W + x]] += 1;
            ++m;
        }
    return m;
}

/* ------------------------------------------------------------------ */
/* Prop. 1: intersection distance, scaled to integers                  */
/* ------------------------------------------------------------------ */

/* int(c_A, c_L) = sum_j min(A[j]/|A|, L[j]/|L|); multiplied by |A||L| it is
 * S(A,L) = sum_j min(A[j]*|L|, L[j]*|A|), an integer. */
static i128 scaled_intersection(const int64_t *A, int64_t sA, const int64_t *Lh, int64_t m, int nbins)
{
    i128 S = 0;
    for (int j = 0; j < nbins; ++j) {
        i128 a = (i128)A[j] * m, l = (i128)Lh[j] * sA;
        S += a < l ? a : l;
    }
    return S;
}

/* f(n) > f_stay for a block L of |L| = m leaving k, given S_n = S(A_n, L):
 * S_n/|A_n| > S(A_k\L, L)/(|A_k|-|L|) */
static int block_beats_stay(ref_state *st, int k, int n, i128 S_n, const int64_t *Lh, int64_t m)
{
    int64_t *Ar = st->tmp_a;
    const int64_t *Ak = st->hist + (int64_t)k * st->nbins;
    for (int j = 0; j < st->nbins; ++j) Ar[j] = Ak[j] - Lh[j];
    int64_t s_rest = st->size[k] - m;
    i128 S_stay = scaled_intersection(Ar, s_rest, Lh, m, st->nbins);
    return S_n * s_rest > S_stay * st->size[n];
}

/* Block move (Sec. 5.2-5.3, Prop. 1; no G for blocks).  Scores are
 * f(n) = int(c_An, c_L) and f_stay = int(c_{Ak\L}, c_L); the common factor
 * 1/|L| is dropped, so f(n) = S(A_n,L)/|A_n|. Returns the target or -1. */
static int decide_block(ref_state *st, int level, int bx, int by)
{
    int k = unit_label(st, level, bx, by);
    int cand[4];
    int nc = candidates(st, level, bx, by, k, cand);
    if (nc == 0) return -1;                               /* not a boundary unit */
    if (!leaving_keeps_connected(st, level, bx, by, k)) return -1;
    int64_t *Lh = st->tmp_l;
    int64_t m = unit_histogram(st, level, bx, by, Lh);
    int best = -1;
    i128 S_best = 0;
    for (int c = 0; c < nc; ++c) {
        int n = cand[c];
        i128 S = scaled_intersection(st->hist + (int64_t)n * st->nbins, st->size[n], Lh, m, st->nbins);
        /* S/|A_n| > S_best/|A_best| */
        if (best < 0 || S * st->size[best] > S_best * st->size[n]) { best = n; S_best = S; }
    }
    /* R8: strictly better than staying */
    return block_beats_stay(st, k, best, S_best, Lh, m) ? best : -1;
}

/* ------------------------------------------------------------------ */
/* Prop. 2: label-patch counts                                          */
/* ------------------------------------------------------------------ */

static int in_image(const ref_state *st, int x, int y) { return x >= 0 && y >= 0 && x < st->W && y < st->H; }

/* sum over the patches N_i that contain pixel p of b_{N_i}(label), in
 * counts (Z = 9 dropped): the two sides of Prop. 2 are built from it.
 * K_p = { i in image : p in N_i }, N_i = in-image 3x3 around i (R13). */
static int64_t patch_label_count(const ref_state *st, int x, int y, int label, int64_t *Kp)
{
    int64_t G = 0, nK = 0;
    for (int iy = y - 1; iy <= y + 1; ++iy)
        for (int ix = x - 1; ix <= x + 1; ++ix) {
            if (!in_image(st, ix, iy)) continue;
            ++nK;
            for (int qy = iy - 1; qy <= iy + 1; ++qy)
                for (int qx = ix - 1; qx <= ix + 1; ++qx)
                    if (in_image(st, qx, qy) && st->lab[(int64_t)qy * st->W + qx] == label) ++G;
        }
    if (Kp) *Kp = nK;
    return G;
}

/* f(n) > f_stay for pixel (x,y) leaving k, times gamma_den*|A_n|*(|A_k|-1):
 *   gamma_den*D*(A_n[j]*(|A_k|-1) - (A_k[j]-1)*|A_n|)
 *     + gamma_num*(G_n + |K_p| - G_k)*|A_n|*(|A_k|-1) > 0 */
static int pixel_beats_stay(const ref_state *st, int x, int y, int k, int n, int64_t a_n, int64_t s_n, int64_t G_n,
                            int64_t G_k, int64_t Kp)
{
    const int use_g = st->p.patch == 3;
    int j = st->bin[(int64_t)y * st->W + x];
    (void)n;
    int64_t a_k = st->hist[(int64_t)k * st->nbins + j], s_k = st->size[k];
    i128 gain = (i128)st->p.gamma_den * 81 * ((i128)a_n * (s_k - 1) - (i128)(a_k - 1) * s_n)
              + (use_g ? (i128)st->p.gamma_num * (G_n + Kp - G_k) * s_n * (s_k - 1) : 0);
    return gain > 0;
}

/* Pixel move (Sec. 5.3): colour term by one histogram lookup (Fig. 6),
 * boundary term by Prop. 2, combined as in R10:
 *   f(n)    = D * A_n[j]/|A_n|           + gamma * (G_n + |K_p|)
 *   f_stay  = D * (A_k[j]-1)/(|A_k|-1)   + gamma * G_k
 * compared exactly after multiplying by gamma_den and the positive sizes. */
static int edge_frozen(const ref_state *st, int x, int y, int k);

static int decide_pixel_compact(ref_state *st, int x, int y, int k, const int *cand, int nc);

static int decide_pixel(ref_state *st, int x, int y)
{
    int k = st->lab[(int64_t)y * st->W + x];
    int cand[4];
    int nc = candidates(st, 0, x, y, k, cand);
    if (nc == 0) return -1;
    if (!leaving_keeps_connected(st, 0, x, y, k)) return -1;
    if (edge_frozen(st, x, y, k)) return -1;
    if (st->p.compact_prior > 0) return decide_pixel_compact(st, x, y, k, cand, nc);
    const int use_g = st->p.patch == 3;
    const i128 D = 81, gn = st->p.gamma_num, gd = st->p.gamma_den;
    int j = st->bin[(int64_t)y * st->W + x];
    int64_t Kp = 0;
    int64_t Gk = use_g ? patch_label_count(st, x, y, k, &Kp) : 0;
    int best = -1;
    int64_t a_b = 0, s_b = 1, G_b = 0;
    for (int c = 0; c < nc; ++c) {
        int n = cand[c];
        int64_t a = st->hist[(int64_t)n * st->nbins + j], s = st->size[n];
        int64_t G = use_g ? patch_label_count(st, x, y, n, NULL) : 0;
        if (best >= 0) {
            /* f(n) - f(best) > 0, times gamma_den*|A_n|*|A_best| */
            i128 diff = gd * D * ((i128)a * s_b - (i128)a_b * s) + gn * (i128)(G - G_b) * s * s_b;
            if (!(diff > 0)) continue;
        }
        best = n; a_b = a; s_b = s; G_b = G;
    }
    return pixel_beats_stay(st, x, y, k, best, a_b, s_b, G_b, Gk, Kp) ? best : -1;
}

/* move a whole unit from k to n: relabel its pixels and update the
 * histograms incrementally (the incremental update of Sec. 5.3) */
static void apply_move(ref_state *st, int level, int bx, int by, int k, int n)
{
    for (int y = st->ye[level][by]; y < st->ye[level][by + 1]; ++y)
        for (int x = st->xe[level][bx]; x < st->xe[level][bx + 1]; ++x) {
            int64_t i = (int64_t)y * st->W + x;
            int j = st->bin[i];
            st->lab[i] = n;
            st->hist[(int64_t)k * st->nbins + j] -= 1;
            st->hist[(int64_t)n * st->nbins + j] += 1;
            st->size[k] -= 1;
            st->size[n] += 1;
        }
}

/* ------------------------------------------------------------------ */
/* edge snapping (R18)                                                  */
/* ------------------------------------------------------------------ */

/* The L1 distance of the colour codes of pixels i and j. */
static int code_l1(const ref_state *st, int64_t i, int64_t j)
{
    int d = 0;
    for (int q = 0; q < 3; ++q) d += abs((int)st->code[3 * i + q] - (int)st->code[3 * j + q]);
    return d;
}

/* A pixel sits on a snapped boundary when one of its 4-neighbours has
 * another label and the two pixels' colour codes differ by at least the
 * edge threshold: such a pixel does not move. */
static int edge_frozen(const ref_state *st, int x, int y, int k)
{
    int tau = st->p.edge_threshold;
    if (tau <= 0) return 0;
    static const int DX[4] = {-1, 1, 0, 0}, DY[4] = {0, 0, -1, 1};
    int64_t i = (int64_t)y * st->W + x;
    for (int d = 0; d < 4; ++d) {
        int qx = x + DX[d], qy = y + DY[d];
        if (qx < 0 || qy < 0 || qx >= st->W || qy >= st->H) continue;
        int64_t j = (int64_t)qy * st->W + qx;
        if (st->lab[j] != k && code_l1(st, i, j) >= tau) return 1;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* means-based pixel updates (R17)                                      */
/* ------------------------------------------------------------------ */

/* sums of the colour codes and of the coordinates of every superpixel */
static void means_recount(ref_state *st)
{
    memset(st->msum, 0, sizeof(int64_t) * (size_t)st->K * 5);
    for (int y = 0; y < st->H; ++y)
        for (int x = 0; x < st->W; ++x) {
            int64_t i = (int64_t)y * st->W + x;
            int64_t *m = st->msum + (int64_t)st->lab[i] * 5;
            m[0] += st->code[3 * i];
            m[1] += st->code[3 * i + 1];
            m[2] += st->code[3 * i + 2];
            m[3] += x;
            m[4] += y;
        }
}

/* SLIC's squared distance of pixel (x,y) to the mean of superpixel `label`
 * (colour codes, then coordinates weighted by (m/S)^2), in IEEE single
 * precision in this order of operations; the mean of a sum S is
 * S * (1/|A|) */
static float means_distance(const ref_state *st, int x, int y, int label)
{
    const int64_t *m = st->msum + (int64_t)label * 5;
    const uint8_t *c = st->code + 3 * ((int64_t)y * st->W + x);
    float r = 1.0f / (float)st->size[label];
    float dc = 0.0f;
    for (int q = 0; q < 3; ++q) {
        float t = (float)c[q] - (float)m[q] * r;
        dc = dc + t * t;
    }
    float gx = (float)x - (float)m[3] * r;
    float gy = (float)y - (float)m[4] * r;
    float ds = gx * gx + gy * gy;
    return dc + st->means_w * ds;
}

/* a boundary pixel that may leave (R5, R7) moves to the candidate with the
 * nearest mean when that is strictly nearer than its own superpixel's mean
 * (which includes the pixel, as SLIC assigns to the nearest centre); ties
 * to the smallest label */
static int decide_pixel_means(ref_state *st, int x, int y)
{
    int k = st->lab[(int64_t)y * st->W + x];
    int cand[4];
    int nc = candidates(st, 0, x, y, k, cand);
    if (nc == 0) return -1;
    if (!leaving_keeps_connected(st, 0, x, y, k)) return -1;
    if (edge_frozen(st, x, y, k)) return -1;
    int best = -1;
    float db = 0.0f;
    for (int c = 0; c < nc; ++c) {
        float d = means_distance(st, x, y, cand[c]);
        if (best < 0 || d < db) {
            best = cand[c];
            db = d;
        }
    }
    return db < means_distance(st, x, y, k) ? best : -1;
}

/* ------------------------------------------------------------------ */
/* compactness prior (R19)                                              */
/* ------------------------------------------------------------------ */

/* The pixel score of one option with the compactness prior, in IEEE single
 * precision in this order: colour term D * a/s (a = the pixel's bin count,
 * s = the size, of the option as it would be: A_n, or A_k without the
 * pixel), boundary term gamma * G (G_n + |K_p| or G_k), minus
 * compact_w * d^2, where d^2 is the squared distance of (x, y) to the
 * centre of gravity of the option's superpixel as it stands (sums from
 * msum over `sc` pixels; the stay option keeps the pixel). */
static float compact_score(const ref_state *st, int x, int y, int label, int64_t a, int64_t s, int64_t sc, int64_t G)
{
    const int64_t *m = st->msum + (int64_t)label * 5;
    float r = 1.0f / (float)sc;
    float gx = (float)x - (float)m[3] * r;
    float gy = (float)y - (float)m[4] * r;
    float d2 = gx * gx + gy * gy;
    float col = (float)a / (float)s;
    float t1 = 81.0f * col;
    float t2 = st->gamma_f * (float)G;
    float t3 = st->compact_w * d2;
    return (t1 + t2) - t3;
}

/* R19: the best candidate by compact_score (ascending, a later one only if
 * strictly higher: ties to the smallest label), accepted if strictly above
 * the stay score.  Centres come from st->msum, recounted at phase start. */
static int decide_pixel_compact(ref_state *st, int x, int y, int k, const int *cand, int nc)
{
    const int use_g = st->p.patch == 3;
    int j = st->bin[(int64_t)y * st->W + x];
    int64_t Kp = 0;
    int64_t Gk = use_g ? patch_label_count(st, x, y, k, &Kp) : 0;
    int best = -1;
    float fb = 0.0f;
    for (int c = 0; c < nc; ++c) {
        int n = cand[c];
        int64_t G = use_g ? patch_label_count(st, x, y, n, NULL) + Kp : 0;
        float f = compact_score(st, x, y, n, st->hist[(int64_t)n * st->nbins + j], st->size[n], st->size[n], G);
        if (best < 0 || f > fb) {
            best = n;
            fb = f;
        }
    }
    float fk = compact_score(st, x, y, k, st->hist[(int64_t)k * st->nbins + j] - 1, st->size[k] - 1, st->size[k], Gk);
    return fb > fk ? best : -1;
}

/* ------------------------------------------------------------------ */
/* the parity schedule (R4, R6)                                         */
/* ------------------------------------------------------------------ */

/* One phase: every unit of the phase is judged against the state at phase
 * start, then all accepted moves are applied.  Returns the number of moves. */
int64_t ref_run_phase(ref_state *st, int level, int phase)
{
    if (level < 0 || level > st->L || phase < 0 || phase > 3) return REF_EINVAL;
    int py = phase >> 1, px = phase & 1;
    int64_t nm = 0;
    if (level == 0 && st->p.compact_prior > 0) means_recount(st); /* R19: centres at phase start */
    for (int by = py; by < st->nby[level]; by += 2)
        for (int bx = px; bx < st->nbx[level]; bx += 2) {
            int n = level == 0 ? decide_pixel(st, bx, by) : decide_block(st, level, bx, by);
            if (n < 0) continue;
            st->moves[3 * nm + 0] = by * st->nbx[level] + bx;
            st->moves[3 * nm + 1] = unit_label(st, level, bx, by);
            st->moves[3 * nm + 2] = n;
            ++nm;
        }
    for (int64_t t = 0; t < nm; ++t) {
        int u = st->moves[3 * t];
        apply_move(st, level, u % st->nbx[level], u / st->nbx[level], st->moves[3 * t + 1], st->moves[3 * t + 2]);
    }
    return nm;
}

/* One means-based pixel phase (R17): the superpixel means are taken at the
 * phase start, every pixel of the phase is judged against them, then all
 * accepted moves are applied.  Returns the number of moves. */
int64_t ref_run_means_phase(ref_state *st, int phase)
{
    if (phase < 0 || phase > 3) return REF_EINVAL;
    int py = phase >> 1, px = phase & 1;
    int64_t nm = 0;
    means_recount(st);
    for (int y = py; y < st->H; y += 2)
        for (int x = px; x < st->W; x += 2) {
            int n = decide_pixel_means(st, x, y);
            if (n < 0) continue;
            st->moves[3 * nm + 0] = y * st->W + x;
            st->moves[3 * nm + 1] = st->lab[(int64_t)y * st->W + x];
            st->moves[3 * nm + 2] = n;
            ++nm;
        }
    for (int64_t t = 0; t < nm; ++t) {
        int u = st->moves[3 * t];
        apply_move(st, 0, u % st->W, u / st->W, st->moves[3 * t + 1], st->moves[3 * t + 2]);
    }
    return nm;
}

/* whole schedule: levels L..1 (blocks), then level 0 (pixels), then the
 * means-based pixel iterations (R17) */
int64_t ref_run(ref_state *st, const uint8_t *rgb, int64_t row_stride)
{
    int rc = ref_init(st, rgb, row_stride);
    if (rc) return rc;
    int64_t total = 0;
    for (int level = st->L; level >= 0; --level)
        for (int it = 0; it < st->p.iters_per_level; ++it)
            for (int phase = 0; phase < 4; ++phase) total += ref_run_phase(st, level, phase);
    for (int it = 0; it < st->p.means_iters; ++it)
        for (int phase = 0; phase < 4; ++phase) total += ref_run_means_phase(st, phase);
    return total;
}

/* R15 anytime termination (Sec. 5.4): the schedule as a list of ops -- the
 * initialisation, then for each level L..1 its 4*iters phases and the
 * descent to the next finer level, then the 4*iters pixel phases, then the
 * output -- run only up to its first `nops` ops (nops >= 1).  With means
 * iterations (R17) the op list has, before the output, one op that starts
 * them and their 4*means_iters phases.  Blocks move
 * their pixels whole here, so descents and the output leave the pixel
 * labels as they are, and the partition after any prefix is the pixel
 * labels.  Returns the number of accepted moves. */
int64_t ref_run_ops(ref_state *st, const uint8_t *rgb, int64_t row_stride, int32_t nops)
{
    if (nops < 1) return REF_EINVAL;
    int rc = ref_init(st, rgb, row_stride);
    if (rc) return rc;
    int64_t total = 0;
    int32_t done = 1; /* the initialisation */
    for (int level = st->L; level >= 0; --level) {
        for (int it = 0; it < st->p.iters_per_level; ++it)
            for (int phase = 0; phase < 4; ++phase) {
                if (done >= nops) return total;
                total += ref_run_phase(st, level, phase);
                ++done;
            }
        if (level > 0) ++done; /* the descent to level-1 */
    }
    if (st->p.means_iters > 0) {
        ++done; /* the start of the means iterations (R17) */
        for (int it = 0; it < st->p.means_iters; ++it)
            for (int phase = 0; phase < 4; ++phase) {
                if (done >= nops) return total;
                total += ref_run_means_phase(st, phase);
                ++done;
            }
    }
    return total; /* the output follows */
}

/* number of ops in the schedule of R15 */
int32_t ref_num_ops(const ref_state *st)
{
    int32_t n = 1 + (st->L + 1) * (4 * st->p.iters_per_level + 1);
    if (st->p.means_iters > 0) n += 1 + 4 * st->p.means_iters;
    return n;
}

/* the means-based decision for one pixel against the current labels
 * (target label, or -1 for no move; test hook) */
int ref_decide_means(ref_state *st, int x, int y)
{
    if (x < 0 || y < 0 || x >= st->W || y >= st->H) return REF_EINVAL;
    means_recount(st);
    return decide_pixel_means(st, x, y);
}

/* ------------------------------------------------------------------ */
/* state access                                                         */
/* ------------------------------------------------------------------ */

void ref_get_labels(const ref_state *st, int32_t *out)
{
    int64_t N = (int64_t)st->W * st->H;
    for (int64_t i = 0; i < N; ++i) out[i] = st->lab[i];
}

void ref_get_bins(const ref_state *st, int32_t *out)
{
    int64_t N = (int64_t)st->W * st->H;
    for (int64_t i = 0; i < N; ++i) out[i] = st->bin[i];
}

void ref_get_hist(const ref_state *st, int64_t *hist_out, int64_t *size_out)
{
    if (hist_out) memcpy(hist_out, st->hist, sizeof(int64_t) * (size_t)st->K * st->nbins);
    if (size_out) memcpy(size_out, st->size, sizeof(int64_t) * (size_t)st->K);
}

/* replace the labels (values in [0,K)) and recount the histograms */
int ref_set_labels(ref_state *st, const int32_t *labels)
{
    int64_t N = (int64_t)st->W * st->H;
    for (int64_t i = 0; i < N; ++i)
        if (labels[i] < 0 || labels[i] >= st->K) return REF_EINVAL;
    for (int64_t i = 0; i < N; ++i) st->lab[i] = labels[i];
    recount_histograms(st);
    return REF_OK;
}

/* sum_{i in K_p} b_{N_i}(label) in counts, and |K_p| */
int64_t ref_patch_label_count(const ref_state *st, int x, int y, int label, int64_t *Kp)
{
    return patch_label_count(st, x, y, label, Kp);
}

/* the parity schedule's decision for one unit against the current state
 * (target label, or -1 for no move) */
int ref_decide(ref_state *st, int level, int bx, int by)
{
    if (level < 0 || level > st->L || bx < 0 || by < 0 || bx >= st->nbx[level] || by >= st->nby[level])
        return REF_EINVAL;
    if (level == 0 && st->p.compact_prior > 0) means_recount(st); /* R19: centres of the current labels */
    return level == 0 ? decide_pixel(st, bx, by) : decide_block(st, level, bx, by);
}

/* ------------------------------------------------------------------ */
/* sequential mode (R14): the paper's proposal order, quality reference */
/* ------------------------------------------------------------------ */

/* SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) */
static uint64_t splitmix64(uint64_t *s)
{
    uint64_t z = (*s += 0x9e3779b97f4a7c15ULL);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* One sweep's visiting order of nu units: the identity shuffled by Fisher
 * and Yates' method in Durstenfeld's form (Knuth, TAOCP vol. 2, 3.4.2,
 * Algorithm P): for u = nu-1 down to 1, swap entry u with a uniformly drawn
 * entry v in [0, u]. */
static void shuffle_units(uint64_t *rng, int32_t *order, int64_t nu)
{
    for (int64_t u = 0; u < nu; ++u) order[u] = (int32_t)u;
    for (int64_t u = nu - 1; u > 0; --u) {
        int64_t v = (int64_t)(splitmix64(rng) % (uint64_t)(u + 1));
        int32_t t = order[u];
        order[u] = order[v];
        order[v] = t;
    }
}

/* the candidate a unit proposes: one of its nc candidates, uniformly */
static int draw_candidate(uint64_t *rng, int nc)
{
    return (int)(splitmix64(rng) % (uint64_t)nc);
}

/* test hooks: the first n draws from state `seed`, the first sweep's
 * visiting order of nu units, and n successive candidate picks among nc,
 * as the sequential mode makes them */
void ref_splitmix64_draws(uint64_t seed, int32_t n, uint64_t *out)
{
    uint64_t rng = seed;
    for (int32_t i = 0; i < n; ++i) out[i] = splitmix64(&rng);
}

void ref_unit_order(uint64_t seed, int32_t nu, int32_t *out)
{
    uint64_t rng = seed;
    shuffle_units(&rng, out, nu);
}

void ref_candidate_picks(uint64_t seed, int32_t nc, int32_t n, int32_t *out)
{
    uint64_t rng = seed;
    for (int32_t i = 0; i < n; ++i) out[i] = draw_candidate(&rng, nc);
}

/* sum over labels of b^2 for the in-image 3x3 patch around (x,y), counts */
static int64_t patch_sum_sq(const ref_state *st, int x, int y)
{
    int labs[9], cnt[9], nl = 0;
    for (int qy = y - 1; qy <= y + 1; ++qy)
        for (int qx = x - 1; qx <= x + 1; ++qx) {
            if (!in_image(st, qx, qy)) continue;
            int l = st->lab[(int64_t)qy * st->W + qx], f = -1;
            for (int t = 0; t < nl; ++t) if (labs[t] == l) f = t;
            if (f < 0) { labs[nl] = l; cnt[nl] = 1; ++nl; } else ++cnt[f];
        }
    int64_t s = 0;
    for (int t = 0; t < nl; ++t) s += (int64_t)cnt[t] * cnt[t];
    return s;
}

/* change of sum_i sum_k b_{N_i}(k)^2 (counts) if unit u moves k -> n */
static int64_t delta_patch_energy(ref_state *st, int level, int bx, int by, int k, int n)
{
    int x0 = st->xe[level][bx], x1 = st->xe[level][bx + 1];
    int y0 = st->ye[level][by], y1 = st->ye[level][by + 1];
    int64_t before = 0, after = 0;
    for (int y = y0 - 1; y <= y1; ++y)
        for (int x = x0 - 1; x <= x1; ++x)
            if (in_image(st, x, y)) before += patch_sum_sq(st, x, y);
    for (int y = y0; y < y1; ++y)
        for (int x = x0; x < x1; ++x) st->lab[(int64_t)y * st->W + x] = n;
    for (int y = y0 - 1; y <= y1; ++y)
        for (int x = x0 - 1; x <= x1; ++x)
            if (in_image(st, x, y)) after += patch_sum_sq(st, x, y);
    for (int y = y0; y < y1; ++y)
        for (int x = x0; x < x1; ++x) st->lab[(int64_t)y * st->W + x] = k;
    return after - before;
}

static i128 sum_sq(const int64_t *A, int nbins)
{
    i128 s = 0;
    for (int j = 0; j < nbins; ++j) s += (i128)A[j] * A[j];
    return s;
}

/* exact energy test: E = H + gamma*G (Eqs. 3, 5, 7) rises strictly when u
 * moves k -> n.  H changes only in A_k and A_n; G changes only in patches
 * touching u.  Everything is multiplied by the positive common denominator
 * (a+m)^2 (b-m)^2 a^2 b^2 * 81 * gamma_den, with a=|A_n|, b=|A_k|, m=|L|. */
static int exact_energy_rises(ref_state *st, int level, int bx, int by, int k, int n)
{
    int64_t *Lh = st->tmp_l, *T = st->tmp_a;
    int64_t m = unit_histogram(st, level, bx, by, Lh);
    const int64_t *An = st->hist + (int64_t)n * st->nbins, *Ak = st->hist + (int64_t)k * st->nbins;
    i128 a = st->size[n], b = st->size[k];
    i128 Qn = sum_sq(An, st->nbins), Qk = sum_sq(Ak, st->nbins);
    for (int j = 0; j < st->nbins; ++j) T[j] = An[j] + Lh[j];
    i128 Qn2 = sum_sq(T, st->nbins);
    for (int j = 0; j < st->nbins; ++j) T[j] = Ak[j] - Lh[j];
    i128 Qk2 = sum_sq(T, st->nbins);
    i128 an2 = (a + m) * (a + m), bk2 = (b - m) * (b - m), a2 = a * a, b2 = b * b;
    i128 dH = Qn2 * bk2 * a2 * b2 + Qk2 * an2 * a2 * b2 - Qn * an2 * bk2 * b2 - Qk * an2 * bk2 * a2;
    i128 gd = st->p.gamma_den, gn = st->p.gamma_num;
    i128 total = 81 * gd * dH;
    if (st->p.patch == 3) {
        i128 dG = delta_patch_energy(st, level, bx, by, k, n);
        total += gn * dG * an2 * bk2 * a2 * b2;
    }
    return total > 0;
}

/* Sequential hill climbing.  accept_mode 0: the parity schedule's proxy
 * rule (Props. 1 and 2, R10; the priors of R18 and R19 are not applied) for
 * the one drawn candidate; 1: exact energy rise
 * (small images only, N <= 1024).  Accepted moves are written to `trace` as
 * (level, unit, k, n) quadruples while room is left.  Returns the number of
 * accepted moves, or a negative error. */
int64_t ref_run_sequential(ref_state *st, const uint8_t *rgb, int64_t row_stride, uint64_t seed, int accept_mode,
                           int32_t *trace, int64_t trace_cap)
{
    if (accept_mode != 0 && accept_mode != 1) return REF_EINVAL;
    if (accept_mode == 1 && (int64_t)st->W * st->H > 1024) return REF_ESIZE;
    int rc = ref_init(st, rgb, row_stride);
    if (rc) return rc;
    uint64_t rng = seed;
    int64_t n_acc = 0;
    int64_t cap_units = (int64_t)st->W * st->H;
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * cap_units);
    if (!order) return REF_ENOMEM;
    for (int level = st->L; level >= 0; --level) {
        int nbx = st->nbx[level], nby = st->nby[level];
        int64_t nu = (int64_t)nbx * nby;
        for (int it = 0; it < st->p.iters_per_level; ++it) {
            shuffle_units(&rng, order, nu);
            for (int64_t t = 0; t < nu; ++t) {
                int bx = order[t] % nbx, by = order[t] / nbx;
                int k = unit_label(st, level, bx, by);
                int cand[4];
                int nc = candidates(st, level, bx, by, k, cand);
                if (nc == 0) continue;
                int n = cand[draw_candidate(&rng, nc)];
                if (!leaving_keeps_connected(st, level, bx, by, k)) continue;
                int ok;
                if (accept_mode == 1) {
                    ok = exact_energy_rises(st, level, bx, by, k, n);
                } else if (level == 0) {
                    /* the pixel rule with only n on offer */
                    const int use_g = st->p.patch == 3;
                    int j = st->bin[(int64_t)by * st->W + bx];
                    int64_t Kp = 0;
                    int64_t Gk = use_g ? patch_label_count(st, bx, by, k, &Kp) : 0;
                    int64_t Gn = use_g ? patch_label_count(st, bx, by, n, NULL) : 0;
                    ok = pixel_beats_stay(st, bx, by, k, n, st->hist[(int64_t)n * st->nbins + j], st->size[n], Gn,
                                          Gk, Kp);
                } else {
                    int64_t *Lh = st->tmp_l;
                    int64_t m = unit_histogram(st, level, bx, by, Lh);
                    i128 S_n = scaled_intersection(st->hist + (int64_t)n * st->nbins, st->size[n], Lh, m, st->nbins);
                    ok = block_beats_stay(st, k, n, S_n, Lh, m);
                }
                if (!ok) continue;
                apply_move(st, level, bx, by, k, n);
                if (trace && n_acc < trace_cap) {
                    trace[4 * n_acc + 0] = level;
                    trace[4 * n_acc + 1] = order[t];
                    trace[4 * n_acc + 2] = k;
                    trace[4 * n_acc + 3] = n;
                }
                ++n_acc;
            }
        }
    }
    free(order);
    return n_acc;
}

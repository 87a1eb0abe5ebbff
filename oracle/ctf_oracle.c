/*
 * ctf_oracle.c -- plain, slow CPU oracle for Collaborative Texture Filtering
 * (Akenine-Moller, Ebelin, Pharr, Wronski: "Collaborative Texture Filtering",
 * HPG 2025, arXiv 2506.17770).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline / reference leg of bench.py load this library.  The product
 * library (paper_2506_17770_gb300) never links, loads or calls it, and the two
 * share no source, header, table or constant generator.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fno-fast-math -shared -fPIC.
 * -ffp-contract=off matters: every float operation below is one IEEE
 * round-to-nearest operation, and the only fused multiply-adds are the explicit
 * fmaf() calls of the filter step.
 *
 * What is here, each with the passage it follows:
 *   - Philox4x32-10 and Philox4x64-10 counter-based generators (Salmon et al.,
 *     "Parallel random numbers: as easy as 1, 2, 3", SC'11), written from the
 *     published round function.  The paper itself names no generator; the STF
 *     fallback draws its two uniforms from Philox4x32-10.
 *   - the bijection h(i,B) (i-th set bit) and its inverse (number of set bits
 *     below t), Sec. 3.3 and Fig. 3.
 *   - exact decode of the project's 4x4-texel block format (the paper only says
 *     "a texel stored in a custom format", Sec. 3): two RGB565 endpoints,
 *     bit-replicated to 8 bits, 4-colour palette (c0, c1, (2c0+c1+1)/3,
 *     (c0+2c1+1)/3), 2-bit index per texel, alpha 255.
 *   - per-pixel 4-tap bilinear (Sec. 3, the filter every success path must
 *     reproduce), one-tap STF (Sec. 3.4 opening: a texel chosen with probability
 *     equal to its filter weight), and the three collaborative algorithms:
 *     List Merge (Sec. 3.1), Box Sampling (Sec. 3.2, Appendix code of Box
 *     Sampling) and Mask Sampling (Sec. 3.3), with edge remapping (supplemental
 *     Sec. 2, "Edge Remapping": producer lane = h(i, A)).
 *
 * Coordinates (Appendix code, first lines): floatCoords = uv*dim - 0.5,
 * upperLeft = floor, st = frac.  Warp tiles are tile_w x tile_h pixels aligned
 * to the frame origin, lane = ty*tile_w + tx.
 */
#include <stdint.h>
#include <stddef.h>
#include <string.h>
#include <stdlib.h>
#include <math.h>

/* ------------------------------------------------------------------------ */
/* Philox (Salmon et al. SC'11).  One round: two multiplications split into  */
/* high and low halves, xor with the other two words and the round key; the  */
/* key is bumped by the Weyl constants between rounds.                        */
/* ------------------------------------------------------------------------ */
#define PHILOX_M4x32_0 0xD2511F53u
#define PHILOX_M4x32_1 0xCD9E8D57u
#define PHILOX_W32_0 0x9E3779B9u
#define PHILOX_W32_1 0xBB67AE85u
#define PHILOX_M4x64_0 0xD2E7470EE14C6C93ull
#define PHILOX_M4x64_1 0xCA5A826395121157ull
#define PHILOX_W64_0 0x9E3779B97F4A7C15ull
#define PHILOX_W64_1 0xBB67AE8584CAA73Bull

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX_W32_0;
            k1 += PHILOX_W32_1;
        }
        uint64_t p0 = (uint64_t)PHILOX_M4x32_0 * (uint64_t)x0;
        uint64_t p1 = (uint64_t)PHILOX_M4x32_1 * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

void oracle_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX_W64_0;
            k1 += PHILOX_W64_1;
        }
        unsigned __int128 p0 = (unsigned __int128)PHILOX_M4x64_0 * x0;
        unsigned __int128 p1 = (unsigned __int128)PHILOX_M4x64_1 * x2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        uint64_t y0 = hi1 ^ x1 ^ k0;
        uint64_t y1 = lo1;
        uint64_t y2 = hi0 ^ x3 ^ k1;
        uint64_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* ------------------------------------------------------------------------ */
/* The bijection of Sec. 3.3 / Fig. 3 over a bit set stored as 32-bit words  */
/* (bit t lives in word t/32, bit t%32).                                      */
/* ------------------------------------------------------------------------ */

/* h(i, B): position of the i-th set bit of B, counting from 0; -1 if B has
 * at most i set bits. */
int oracle_h(const uint32_t *B, int nwords, int i)
{
    int seen = 0;
    for (int t = 0; t < nwords * 32; ++t) {
        if ((B[t / 32] >> (t % 32)) & 1u) {
            if (seen == i)
                return t;
            ++seen;
        }
    }
    return -1;
}

/* h^{-1}(t, B): number of set bits of B strictly below position t. */
int oracle_hinv(const uint32_t *B, int nwords, int t)
{
    int count = 0;
    for (int u = 0; u < t && u < nwords * 32; ++u)
        if ((B[u / 32] >> (u % 32)) & 1u)
            ++count;
    return count;
}

static int popcount_words(const uint32_t *B, int nwords)
{
    int c = 0;
    for (int t = 0; t < nwords * 32; ++t)
        c += (int)((B[t / 32] >> (t % 32)) & 1u);
    return c;
}

/* ------------------------------------------------------------------------ */
/* Exact decode of the 4x4-texel block format.                               */
/* Block (bx, by) of a Wt x Ht texture sits at byte 8*(by*(Wt/4)+bx); bytes  */
/* 0-1 = c0 (RGB565, little endian), 2-3 = c1, 4-7 = 32 index bits; texel    */
/* (x&3, y&3) uses index bits 2*(4*(y&3)+(x&3)) and the next one.            */
/* ------------------------------------------------------------------------ */
static void expand565(unsigned c, int rgb[3])
{
    unsigned r5 = (c >> 11) & 31u, g6 = (c >> 5) & 63u, b5 = c & 31u;
    rgb[0] = (int)((r5 << 3) | (r5 >> 2));
    rgb[1] = (int)((g6 << 2) | (g6 >> 4));
    rgb[2] = (int)((b5 << 3) | (b5 >> 2));
}

/* Decode texel (x, y) to RGBA8.  Coordinates are clamped to the texture
 * (clamp-to-edge): the appendix omits clamping, and this is the one place the
 * oracle applies it. */
void oracle_decode_rgba8(const uint8_t *blocks, int Wt, int Ht, int x, int y, uint8_t rgba[4])
{
    if (x < 0) x = 0;
    if (x > Wt - 1) x = Wt - 1;
    if (y < 0) y = 0;
    if (y > Ht - 1) y = Ht - 1;
    size_t bx = (size_t)(x / 4), by = (size_t)(y / 4), nbx = (size_t)(Wt / 4);
    const uint8_t *b = blocks + 8 * (by * nbx + bx);
    unsigned c0 = (unsigned)b[0] | ((unsigned)b[1] << 8);
    unsigned c1 = (unsigned)b[2] | ((unsigned)b[3] << 8);
    uint32_t bits = (uint32_t)b[4] | ((uint32_t)b[5] << 8) | ((uint32_t)b[6] << 16) | ((uint32_t)b[7] << 24);
    int texel = 4 * (y % 4) + (x % 4);
    int sel = (int)((bits >> (2 * texel)) & 3u);
    int e0[3], e1[3];
    expand565(c0, e0);
    expand565(c1, e1);
    for (int ch = 0; ch < 3; ++ch) {
        int v;
        switch (sel) {
        case 0: v = e0[ch]; break;
        case 1: v = e1[ch]; break;
        case 2: v = (2 * e0[ch] + e1[ch] + 1) / 3; break;
        default: v = (e0[ch] + 2 * e1[ch] + 1) / 3; break;
        }
        rgba[ch] = (uint8_t)v;
    }
    rgba[3] = 255;
}

/* RGBA8 -> float, each channel v/255 correctly rounded (IEEE division). */
static void decode_texel_f32(const uint8_t *blocks, int Wt, int Ht, int x, int y, float out[4])
{
    uint8_t c[4];
    oracle_decode_rgba8(blocks, Wt, Ht, x, y, c);
    for (int k = 0; k < 4; ++k)
        out[k] = (float)c[k] / 255.0f;
}

/* ------------------------------------------------------------------------ */
/* Texel sources.  The filter below asks a source for texel values; the     */
/* exact source is the block decode, the learned source (ctf_oracle_mlp.c)  */
/* is the FP64 MLP over the latent grids.                                    */
/* ------------------------------------------------------------------------ */
typedef struct {
    int kind;                 /* 0 = exact blocks, 1 = learned (FP64 MLP) */
    int Wt, Ht;
    const uint8_t *blocks;    /* kind 0 */
    const void *mlp;          /* kind 1: struct oracle_mlp (ctf_oracle_mlp.c) */
} texel_source;

void oracle_mlp_texel_f64(const void *mlp, int Wt, int Ht, int x, int y, double out[4]);

static void fetch_texel(const texel_source *src, int x, int y, float vf[4], double vd[4])
{
    if (src->kind == 0) {
        decode_texel_f32(src->blocks, src->Wt, src->Ht, x, y, vf);
        for (int k = 0; k < 4; ++k)
            vd[k] = (double)vf[k];
    } else {
        int xc = x < 0 ? 0 : (x > src->Wt - 1 ? src->Wt - 1 : x);
        int yc = y < 0 ? 0 : (y > src->Ht - 1 ? src->Ht - 1 : y);
        oracle_mlp_texel_f64(src->mlp, src->Wt, src->Ht, xc, yc, vd);
        for (int k = 0; k < 4; ++k)
            vf[k] = (float)vd[k];
    }
}

/* ------------------------------------------------------------------------ */
/* Per-pixel setup (Appendix code, first lines; minification rule).          */
/* ------------------------------------------------------------------------ */
typedef struct {
    int active;
    int px, py;       /* pixel in the frame passed in */
    int ry;           /* its row in the full view (py + the band's first row): STF counter word 1 */
    int ulx, uly;     /* upper-left integer texel of the 2x2 footprint */
    float s, t;       /* local coordinates in the 2x2 footprint, in [0,1) */
    int minified;
} pixel_setup;

/* Range guard: |uv*dim - 0.5| must stay below 2^22 so that floor() and the
 * integer bounding box never overflow.  Pixels outside it, with non-finite
 * UVs, outside the frame or with coverage 0 are inactive. */
#define COORD_LIMIT 4194304.0f

static void setup_pixel(const float *uv, const float *jac, const uint8_t *cov, int W, int H,
                        int Wt, int Ht, int px, int py, pixel_setup *p)
{
    memset(p, 0, sizeof(*p));
    p->px = px;
    p->py = py;
    if (px >= W || py >= H)
        return;
    size_t idx = (size_t)py * (size_t)W + (size_t)px;
    if (cov && cov[idx] == 0)
        return;
    float u = uv[2 * idx + 0], v = uv[2 * idx + 1];
    float fW = (float)Wt, fH = (float)Ht;
    float xf = u * fW;         /* one rounding */
    xf = xf - 0.5f;            /* one rounding */
    float yf = v * fH;
    yf = yf - 0.5f;
    if (!(fabsf(xf) < COORD_LIMIT) || !(fabsf(yf) < COORD_LIMIT))
        return; /* also rejects NaN */
    float fx = floorf(xf), fy = floorf(yf);
    p->ulx = (int)fx;
    p->uly = (int)fy;
    p->s = xf - fx;
    p->t = yf - fy;
    /* Minification: rho_x^2 = (du/dx*Wt)^2 + (dv/dx*Ht)^2, rho_y^2 likewise;
     * the pixel is minified unless both are <= 1 (NaN counts as minified). */
    float a = jac[4 * idx + 0] * fW;
    float b = jac[4 * idx + 1] * fH;
    float c = jac[4 * idx + 2] * fW;
    float d = jac[4 * idx + 3] * fH;
    float aa = a * a, bb = b * b, cc = c * c, dd = d * d;
    float rx = aa + bb;
    float ry = cc + dd;
    p->minified = !(rx <= 1.0f && ry <= 1.0f);
    p->active = 1;
}

/* Bilinear weights for taps k = (k%2, k/2): (1-s)(1-t), s(1-t), (1-s)t, st.
 * Appendix code names computeBilinearWeights without defining it. */
static void bilinear_weights(float s, float t, float w[4])
{
    float os = 1.0f - s, ot = 1.0f - t;
    w[0] = os * ot;
    w[1] = s * ot;
    w[2] = os * t;
    w[3] = s * t;
}


/* One-tap STF texel choice: Philox4x32-10 with counter (px, py, view, 0) and
 * key (seed low, seed high); xi = (r >> 8) * 2^-24; the right neighbour is
 * taken when xi0 < s, the lower one when xi1 < t.  Each of the 4 taps is thus
 * chosen with probability equal to its bilinear weight (up to the 2^-24
 * quantisation of xi). */
void oracle_stf_offset(int px, int py, int view, uint64_t seed, float s, float t, int *dx, int *dy)
{
    uint32_t ctr[4] = {(uint32_t)px, (uint32_t)py, (uint32_t)view, 0u};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    uint32_t r[4];
    oracle_philox4x32_10(ctr, key, r);
    float xi0 = (float)(r[0] >> 8) * 0x1p-24f;
    float xi1 = (float)(r[1] >> 8) * 0x1p-24f;
    *dx = xi0 < s ? 1 : 0;
    *dy = xi1 < t ? 1 : 0;
}

/*
 * Bicubic filters (Sec. 4.2): the 4x4 texels from one left of and above the
 * upper-left texel of the bilinear footprint, separable weights w_x(s) w_y(t)
 * with s, t the same fractions.  Cubic B-spline:
 *   ((1-f)^3, 3f^3 - 6f^2 + 4, -3f^3 + 3f^2 + 3f + 1, f^3) / 6;
 * Catmull-Rom (cubic convolution, a = -1/2):
 *   (2f^2 - f^3 - f, 3f^3 - 5f^2 + 2, -3f^3 + 4f^2 + f, f^3 - f^2) / 2;
 * each term a single round-to-nearest FP32 operation in the order written.
 */
enum { FILTER_BILINEAR = 0, FILTER_BSPLINE = 1, FILTER_CATMULL_ROM = 2 };

static int filter_side(int filter) { return filter == FILTER_BILINEAR ? 2 : 4; }

static void cubic_weights(int filter, float f, float w[4])
{
    float f2 = f * f, f3 = f2 * f;
    if (filter == FILTER_BSPLINE) {
        float u = 1.0f - f;
        w[0] = ((u * u) * u) / 6.0f;
        w[1] = ((3.0f * f3 - 6.0f * f2) + 4.0f) / 6.0f;
        w[2] = (((-3.0f * f3 + 3.0f * f2) + 3.0f * f) + 1.0f) / 6.0f;
        w[3] = f3 / 6.0f;
    } else {
        w[0] = 0.5f * ((2.0f * f2 - f3) - f);
        w[1] = 0.5f * ((3.0f * f3 - 5.0f * f2) + 2.0f);
        w[2] = 0.5f * ((-3.0f * f3 + 4.0f * f2) + f);
        w[3] = 0.5f * (f3 - f2);
    }
}

/* Weights of the F x F taps k = j F + i (tap (ox + i, oy + j)); returns F*F. */
static int filter_weights(int filter, float s, float t, float *w)
{
    if (filter == FILTER_BILINEAR) {
        bilinear_weights(s, t, w);
        return 4;
    }
    float wx[4], wy[4];
    cubic_weights(filter, s, wx);
    cubic_weights(filter, t, wy);
    for (int j = 0; j < 4; ++j)
        for (int i = 0; i < 4; ++i)
            w[4 * j + i] = wx[i] * wy[j];
    return 16;
}

/* acc = fma(w_k, p_k, acc) from 0 over the n taps in order (FP32), or the
 * weighted sum in double. */
static void filter_n(int n, const float *w, float p[][4], double pd[][4], int fp64, float out[4], double outd[4])
{
    for (int ch = 0; ch < 4; ++ch) {
        if (!fp64) {
            float acc = 0.0f;
            for (int k = 0; k < n; ++k)
                acc = fmaf(w[k], p[k][ch], acc);
            out[ch] = acc;
            outd[ch] = (double)acc;
        } else {
            double acc = 0.0;
            for (int k = 0; k < n; ++k)
                acc += (double)w[k] * pd[k][ch];
            outd[ch] = acc;
            out[ch] = (float)acc;
        }
    }
}

/* One tap of 4 drawn with probability |w_i| / sum |w| by xi in [0, 1):
 * cumulative sums c in tap order, the first i with xi * S < c_i.  *g is
 * S with the sign of w_i. */
static int pick_tap(const float w[4], float xi, float *g)
{
    float a0 = fabsf(w[0]), a1 = fabsf(w[1]), a2 = fabsf(w[2]), a3 = fabsf(w[3]);
    float c0 = a0, c1 = c0 + a1, c2 = c1 + a2, S = c2 + a3;
    float tsel = xi * S;
    int i = tsel < c0 ? 0 : (tsel < c1 ? 1 : (tsel < c2 ? 2 : 3));
    *g = w[i] < 0.0f ? -S : S;
    return i;
}

/* ------------------------------------------------------------------------ */
/* Algorithms and per-tile outcome codes (shared numbering with the public  */
/* interface; the numbers are the only thing the two sides agree on).       */
/* ------------------------------------------------------------------------ */
enum { ALG_4TAP = 0, ALG_STF = 1, ALG_LIST_MERGE = 2, ALG_BOX = 3, ALG_MASK = 4 };
enum { PATH_EMPTY = 0, PATH_SUCCESS = 1, PATH_FALLBACK_BUDGET = 2, PATH_FALLBACK_MINIFIED = 3, PATH_DIRECT = 4 };

typedef struct {
    int64_t tiles_total, tiles_empty, tiles_direct, tiles_success;
    int64_t tiles_fallback_budget, tiles_fallback_minified;
    int64_t pixels_active, texel_evals;
} oracle_stats;

/* Output for one active lane on the STF path: its own STF texel, count 1.
 * Bilinear: the separable Bernoulli draw.  Bicubic: per axis the tap drawn
 * with probability |w| / sum |w| (pick_tap, xi0 for x and xi1 for y of the
 * same Philox draw); the B-spline returns the texel, Catmull-Rom the texel
 * times sign(w_x) S_x times sign(w_y) S_y (one-sample estimate of the
 * filter with negative lobes; positivization would need two texels). */
static void stf_lane(const texel_source *src, const pixel_setup *p, int filter, int view, uint64_t seed,
                     int fp64, float *out, double *outd, uint8_t *evals, size_t idx, int *tx, int *ty)
{
    float gx = 1.0f, gy = 1.0f;
    if (filter == FILTER_BILINEAR) {
        int dx, dy;
        oracle_stf_offset(p->px, p->ry, view, seed, p->s, p->t, &dx, &dy);
        *tx = p->ulx + dx;
        *ty = p->uly + dy;
    } else {
        uint32_t ctr[4] = {(uint32_t)p->px, (uint32_t)p->ry, (uint32_t)view, 0u};
        uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
        uint32_t r[4];
        oracle_philox4x32_10(ctr, key, r);
        float wx[4], wy[4];
        cubic_weights(filter, p->s, wx);
        cubic_weights(filter, p->t, wy);
        int i = pick_tap(wx, (float)(r[0] >> 8) * 0x1p-24f, &gx);
        int j = pick_tap(wy, (float)(r[1] >> 8) * 0x1p-24f, &gy);
        *tx = p->ulx - 1 + i;
        *ty = p->uly - 1 + j;
    }
    float vf[4];
    double vd[4];
    fetch_texel(src, *tx, *ty, vf, vd);
    const int scale = filter == FILTER_CATMULL_ROM;
    for (int ch = 0; ch < 4; ++ch) {
        float of = fp64 ? (float)vd[ch] : vf[ch];
        double od = fp64 ? vd[ch] : (double)vf[ch];
        if (scale) {
            of = (vf[ch] * gx) * gy;
            od = fp64 ? (vd[ch] * (double)gx) * (double)gy : (double)of;
            if (fp64) of = (float)od;
        }
        if (out) out[4 * idx + ch] = of;
        if (outd) outd[4 * idx + ch] = od;
    }
    evals[idx] = 1;
}

/* Set of unique texel coordinates, kept in insertion order (a wave's 4x4
 * footprints hold at most 32 x 16 texels). */
typedef struct {
    int n;
    int x[512], y[512];
} texel_list;

static int list_find(const texel_list *L, int x, int y)
{
    for (int i = 0; i < L->n; ++i)
        if (L->x[i] == x && L->y[i] == y)
            return i;
    return -1;
}

/*
 * Distinct texels evaluated by a group of consecutive tiles, after clamping
 * to the texture (a group of 8 tiles evaluates at most 8 x 32 texels).  This
 * is the count of the shared-memory extension Sec. 6 proposes, in which a
 * group of warps evaluates each texel once.
 */
typedef struct {
    int n;
    int x[256], y[256];
} group_set;

static void group_note(group_set *G, const texel_source *src, int x, int y)
{
    if (!G)
        return;
    int xc = x < 0 ? 0 : (x > src->Wt - 1 ? src->Wt - 1 : x);
    int yc = y < 0 ? 0 : (y > src->Ht - 1 ? src->Ht - 1 : y);
    for (int i = 0; i < G->n; ++i)
        if (G->x[i] == xc && G->y[i] == yc)
            return;
    if (G->n < 256) {
        G->x[G->n] = xc;
        G->y[G->n] = yc;
        G->n++;
    }
}

/*
 * Eq. 2 with the wave of 32 lanes replaced by the na active lanes: the
 * source lane (index among the active lanes) whose footprint remaining lane
 * c (n <= c < na) draws from, l = round((na-1)(c-n) / (na-1-n)) rounded half
 * up, and l = 0 when a single lane remains (na-1 = n, where the equation
 * reads 0/0).  Returns -1 for arguments outside that range.
 */
int oracle_cplus_source(int na, int n, int c)
{
    if (na < 1 || na > 32 || n < 0 || n >= na || c < n || c >= na)
        return -1;
    const int den = na - 1 - n;
    return den == 0 ? 0 : (2 * (na - 1) * (c - n) + den) / (2 * den);
}

/*
 * Fallbacks C and C+ (Sec. 3.4, "New Fallback Methods") for a magnified tile
 * whose texel set does not fit the budget.  mode 1 = C, 2 = C+.
 *
 * Every active lane draws its one-tap STF texel.  C: every active lane
 * produces its STF texel.  C+: the distinct STF texels U (in the order of
 * the first active lane that draws each; the order changes no output) are
 * produced by the first |U| = n active lanes, and each remaining active lane
 * c (index among the active lanes, n <= c < na) takes the footprint of
 * active lane l = round_half_up((na-1)(c-n)/(na-1-n)) (l = 0 when na-1 = n;
 * eq. 2 with 32 replaced by the number of active lanes na) and produces one
 * of its taps with nonzero weight outside U, chosen with probability
 * proportional to the weights by xi2 = (r2 >> 8) 2^-24, the third word of
 * the lane's own STF draw; a lane whose source has no such tap produces
 * nothing.  Then every active pixel filters with the N distinct texels of
 * its footprint that have nonzero weight and were produced (eq. 1):
 *   N = all nonzero-weight taps: the 4-tap filter (zero-weight taps add
 *       nothing to it), i.e. exact bilinear;
 *   N = 1: that texel;
 *   else: c = fma(1 - S_w, S_p / N, S_wp) per channel, with S_wp the fma
 *       chain of w_k p_k, S_w the sum of w_k and S_p the sum of p_k over the
 *       produced taps in tap order (FP32; FP64 mode in double).
 * Counts: 1 per producing lane.
 */
static void fallback_c(const texel_source *src, const pixel_setup *lane, uint32_t A, int mode, int view,
                       uint64_t seed, int fp64, int W, float *out, double *outd, uint8_t *evals, group_set *G)
{
    int act[32], na = 0;
    for (int l = 0; l < 32; ++l)
        if ((A >> l) & 1u) act[na++] = l;
    int sx[32], sy[32];
    float xi2[32];
    for (int i = 0; i < na; ++i) {
        const pixel_setup *p = &lane[act[i]];
        uint32_t ctr[4] = {(uint32_t)p->px, (uint32_t)p->ry, (uint32_t)view, 0u};
        uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
        uint32_t r[4];
        oracle_philox4x32_10(ctr, key, r);
        float xi0 = (float)(r[0] >> 8) * 0x1p-24f, xi1 = (float)(r[1] >> 8) * 0x1p-24f;
        xi2[i] = (float)(r[2] >> 8) * 0x1p-24f;
        sx[i] = p->ulx + (xi0 < p->s ? 1 : 0);
        sy[i] = p->uly + (xi1 < p->t ? 1 : 0);
    }
    /* produced texels: coordinates and values (a texel may appear twice) */
    int pn = 0, qx[32], qy[32];
    float qv[32][4];
    double qd[32][4];
#define PRODUCE(l_, x_, y_)                                                   \
    do {                                                                      \
        qx[pn] = (x_);                                                        \
        qy[pn] = (y_);                                                        \
        fetch_texel(src, qx[pn], qy[pn], qv[pn], qd[pn]);                     \
        group_note(G, src, qx[pn], qy[pn]);                                   \
        evals[(size_t)lane[l_].py * W + lane[l_].px] = 1;                     \
        pn++;                                                                 \
    } while (0)
    if (mode == 1) {
        for (int i = 0; i < na; ++i) PRODUCE(act[i], sx[i], sy[i]);
    } else {
        int ux[32], uy[32], n = 0;
        for (int i = 0; i < na; ++i) {
            int seen = 0;
            for (int j = 0; j < n; ++j) seen |= ux[j] == sx[i] && uy[j] == sy[i];
            if (!seen) {
                ux[n] = sx[i];
                uy[n] = sy[i];
                n++;
            }
        }
        for (int i = 0; i < n; ++i) PRODUCE(act[i], ux[i], uy[i]);
        for (int c = n; c < na; ++c) {
            const int l = oracle_cplus_source(na, n, c);
            const pixel_setup *q = &lane[act[l]];
            float w[4];
            bilinear_weights(q->s, q->t, w);
            int cand[4], nc = 0;
            for (int k = 0; k < 4; ++k) {
                if (!(w[k] > 0.0f)) continue;
                int tx = q->ulx + k % 2, ty = q->uly + k / 2, inu = 0;
                for (int j = 0; j < n; ++j) inu |= ux[j] == tx && uy[j] == ty;
                if (!inu) cand[nc++] = k;
            }
            if (nc == 0) continue;
            float wc = 0.0f;
            for (int j = 0; j < nc; ++j) wc = wc + w[cand[j]];
            const float tsel = xi2[c] * wc;
            int pick = cand[nc - 1];
            float run = 0.0f;
            for (int j = 0; j < nc; ++j) {
                run = run + w[cand[j]];
                if (tsel < run) {
                    pick = cand[j];
                    break;
                }
            }
            PRODUCE(act[c], q->ulx + pick % 2, q->uly + pick / 2);
        }
    }
#undef PRODUCE
    /* eq. 1 for every active pixel */
    for (int i = 0; i < na; ++i) {
        const pixel_setup *p = &lane[act[i]];
        size_t idx = (size_t)p->py * W + p->px;
        float w[4];
        bilinear_weights(p->s, p->t, w);
        int nz = 0, N = 0, at[4];
        for (int k = 0; k < 4; ++k) {
            at[k] = -1;
            if (!(w[k] > 0.0f)) continue;
            nz++;
            for (int j = 0; j < pn; ++j)
                if (qx[j] == p->ulx + k % 2 && qy[j] == p->uly + k / 2) {
                    at[k] = j;
                    break;
                }
            if (at[k] >= 0) N++;
        }
        for (int ch = 0; ch < 4; ++ch) {
            float o;
            double od;
            if (N == 1) {
                int j = -1;
                for (int k = 0; k < 4; ++k)
                    if (at[k] >= 0) j = at[k];
                o = qv[j][ch];
                od = qd[j][ch];
            } else if (!fp64) {
                float swp = 0.0f, sw = 0.0f, sp = 0.0f;
                for (int k = 0; k < 4; ++k) {
                    if (at[k] < 0) continue;
                    swp = fmaf(w[k], qv[at[k]][ch], swp);
                    sw = sw + w[k];
                    sp = sp + qv[at[k]][ch];
                }
                o = N == nz ? swp : fmaf(1.0f - sw, sp / (float)N, swp);
                od = (double)o;
            } else {
                double swp = 0.0, sw = 0.0, sp = 0.0;
                for (int k = 0; k < 4; ++k) {
                    if (at[k] < 0) continue;
                    swp += (double)w[k] * qd[at[k]][ch];
                    sw += (double)w[k];
                    sp += qd[at[k]][ch];
                }
                od = N == nz ? swp : swp + (1.0 - sw) * sp / (double)N;
                o = (float)od;
            }
            if (out) out[4 * idx + ch] = o;
            if (outd) outd[4 * idx + ch] = od;
        }
    }
}


/*
 * oracle_filter_ex: filter one frame.
 *   src            texel source (exact blocks or learned)
 *   uv   [H][W][2] float, jac [H][W][4] float = (du/dx, dv/dx, du/dy, dv/dy)
 *   cov  [H][W] uint8 or NULL
 *   out  [H][W][4] float (FP32 result; may be NULL), outd [H][W][4] double (may be NULL)
 *   evals[H][W] uint8 per-pixel texel evaluations
 *   tile_path / tile_n: per tile outcome code and texel-set size (may be NULL)
 *   filter         0 bilinear (2x2), 1 cubic B-spline, 2 Catmull-Rom (4x4,
 *                  Sec. 4.2); the bicubic ones with one texel per lane and
 *                  the one-tap STF fallback only
 *   tpl            texels a lane may produce, 1 or 2 (Sec. 5: "more than
 *                  one texel per lane"); budget up to 32 * tpl
 *   fallback       0: over-budget tiles take one-tap STF; 1: fallback C;
 *                  2: fallback C+ (Sec. 3.4); minified tiles always STF
 *   group_tiles    0, or the size of the tile groups (consecutive tile
 *                  indices, at most 8) whose distinct evaluated texels
 *                  stats[8] counts; 4TAP is never grouped
 *   y0             row of the full view at which this frame starts (a band
 *                  of whole tile rows: y0 a multiple of tile_h); it only
 *                  enters the STF counters, which are per pixel of the view
 *   stats[9]       tiles_total, tiles_empty, tiles_direct, tiles_success,
 *                  tiles_fallback_budget, tiles_fallback_minified,
 *                  pixels_active, texel_evals (sum of evals), and the
 *                  grouped distinct-texel count (texel_evals if ungrouped)
 * Returns 0 on success, -1 on bad arguments.
 */
static int oracle_filter_ex(const texel_source *src, const float *uv, const float *jac, const uint8_t *cov,
                            int W, int H, int view, int alg, uint64_t seed, int tile_w, int tile_h,
                            int budget, int mask_dim, int edge_remap, int group_tiles, int fallback, int tpl,
                            int filter, int y0, int fp64, float *out, double *outd, uint8_t *evals,
                            int32_t *tile_path, int32_t *tile_n, int64_t *stats_out)
{
    if (y0 < 0 || y0 % tile_h != 0)
        return -1;
    if (tpl != 1 && tpl != 2)
        return -1;
    if (filter < 0 || filter > 2 || (filter != FILTER_BILINEAR && (fallback != 0 || tpl != 1)))
        return -1;
    const int F = filter_side(filter), off = F == 4 ? 1 : 0;
    if (fallback < 0 || fallback > 2)
        return -1;
    if (W < 0 || H < 0 || tile_w <= 0 || tile_h <= 0 || tile_w * tile_h != 32)
        return -1;
    if (group_tiles < 0 || group_tiles > 8)
        return -1;
    if (alg < 0 || alg > 4 || budget < 1 || budget > 32 * tpl)
        return -1;
    if (alg == ALG_MASK && mask_dim != 16 && mask_dim != 11)
        return -1;
    oracle_stats st;
    memset(&st, 0, sizeof(st));
    int tiles_x = (W + tile_w - 1) / tile_w, tiles_y = (H + tile_h - 1) / tile_h;
    /* groups of group_tiles consecutive tiles (tile index order); 4TAP is
       never grouped */
    const int grouped = group_tiles > 0 && alg != ALG_4TAP;
    group_set G;
    G.n = 0;
    int cur_group = 0;
    int64_t unique = 0;
    for (int by = 0; by < tiles_y; ++by) {
        for (int bx = 0; bx < tiles_x; ++bx) {
            int tile_id = by * tiles_x + bx;
            if (grouped && tile_id / group_tiles != cur_group) {
                unique += G.n;
                G.n = 0;
                cur_group = tile_id / group_tiles;
            }
            pixel_setup lane[32];
            uint32_t A = 0;
            int any_minified = 0;
            for (int l = 0; l < 32; ++l) {
                int px = bx * tile_w + l % tile_w, py = by * tile_h + l / tile_w;
                setup_pixel(uv, jac, cov, W, H, src->Wt, src->Ht, px, py, &lane[l]);
                lane[l].ry = py + y0;
                if (lane[l].active) {
                    A |= 1u << l;
                    any_minified |= lane[l].minified;
                    st.pixels_active++;
                }
                if (px < W && py < H) {
                    size_t idx = (size_t)py * W + px;
                    evals[idx] = 0;
                    for (int ch = 0; ch < 4; ++ch) {
                        if (out) out[4 * idx + ch] = 0.0f;
                        if (outd) outd[4 * idx + ch] = 0.0;
                    }
                }
            }
            st.tiles_total++;
            int path = PATH_EMPTY, nset = 0;
            if (A == 0) {
                st.tiles_empty++;
                if (tile_path) tile_path[tile_id] = PATH_EMPTY;
                if (tile_n) tile_n[tile_id] = 0;
                continue;
            }
            int nactive = popcount_words(&A, 1);

            if (alg == ALG_4TAP || alg == ALG_STF) {
                path = PATH_DIRECT;
                for (int l = 0; l < 32; ++l) {
                    if (!lane[l].active) continue;
                    const pixel_setup *p = &lane[l];
                    size_t idx = (size_t)p->py * W + p->px;
                    if (alg == ALG_STF) {
                        int tx, ty;
                        stf_lane(src, p, filter, view, seed, fp64, out, outd, evals, idx, &tx, &ty);
                        group_note(grouped ? &G : NULL, src, tx, ty);
                    } else {
                        float w[16], pv[16][4], o[4];
                        double pd[16][4], od[4];
                        const int nt = filter_weights(filter, p->s, p->t, w);
                        for (int k = 0; k < nt; ++k)
                            fetch_texel(src, p->ulx - off + k % F, p->uly - off + k / F, pv[k], pd[k]);
                        filter_n(nt, w, pv, pd, fp64, o, od);
                        for (int ch = 0; ch < 4; ++ch) {
                            if (out) out[4 * idx + ch] = o[ch];
                            if (outd) outd[4 * idx + ch] = od[ch];
                        }
                        evals[idx] = (uint8_t)nt;
                    }
                }
                st.tiles_direct++;
                if (tile_path) tile_path[tile_id] = path;
                if (tile_n) tile_n[tile_id] = alg == ALG_STF ? nactive : F * F * nactive;
                continue;
            }

            /* Collaborative algorithms.  Step 1: collect the wave's needs. */
            texel_list L;
            L.n = 0;
            int fits = 1;
            if (any_minified) {
                fits = 0;
                path = PATH_FALLBACK_MINIFIED;
                nset = -1;
            } else {
                /* Wave bounding box: min of upper-left corners, max of
                 * upper-left + (1,1) (Appendix code of Box Sampling). */
                int minx = 0, miny = 0, maxx = 0, maxy = 0, first = 1;
                for (int l = 0; l < 32; ++l) {
                    if (!lane[l].active) continue;
                    int ux = lane[l].ulx - off, uy = lane[l].uly - off;
                    if (first || ux < minx) minx = ux;
                    if (first || uy < miny) miny = uy;
                    if (first || ux + F - 1 > maxx) maxx = ux + F - 1;
                    if (first || uy + F - 1 > maxy) maxy = uy + F - 1;
                    first = 0;
                }
                int64_t bw = (int64_t)maxx - minx + 1, bh = (int64_t)maxy - miny + 1;
                if (alg == ALG_BOX) {
                    /* n = area of the bounding box; texel i = UL + (i % w, i / w). */
                    int64_t area = bw * bh;
                    nset = area > 0x7fffffff ? 0x7fffffff : (int)area;
                    if (area <= budget) {
                        for (int i = 0; i < (int)area; ++i) {
                            L.x[L.n] = minx + (int)(i % bw);
                            L.y[L.n] = miny + (int)(i / bw);
                            L.n++;
                        }
                    } else {
                        fits = 0;
                    }
                } else if (alg == ALG_MASK) {
                    /* Bit (dy*M + dx) for each of the 2x2 texels of each lane,
                     * OR over the wave; texel i = the i-th set bit, h(i, B). */
                    int M = mask_dim;
                    if (bw > M || bh > M) {
                        fits = 0;
                        nset = -1;
                    } else {
                        uint32_t B[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                        int nwords = (M * M + 31) / 32;
                        for (int l = 0; l < 32; ++l) {
                            if (!lane[l].active) continue;
                            int dx = lane[l].ulx - off - minx, dy = lane[l].uly - off - miny;
                            for (int k = 0; k < F * F; ++k) {
                                int tb = (dy + k / F) * M + (dx + k % F);
                                B[tb / 32] |= 1u << (tb % 32);
                            }
                        }
                        nset = popcount_words(B, nwords);
                        if (nset <= budget) {
                            for (int i = 0; i < nset; ++i) {
                                int tb = oracle_h(B, nwords, i);
                                L.x[L.n] = minx + tb % M;
                                L.y[L.n] = miny + tb / M;
                                L.n++;
                            }
                        } else {
                            fits = 0;
                        }
                    }
                } else { /* ALG_LIST_MERGE: the exact set union of all 2x2 lists. */
                    for (int l = 0; l < 32; ++l) {
                        if (!lane[l].active) continue;
                        for (int k = 0; k < F * F; ++k) {
                            int x = lane[l].ulx - off + k % F, y = lane[l].uly - off + k / F;
                            if (list_find(&L, x, y) < 0) {
                                L.x[L.n] = x;
                                L.y[L.n] = y;
                                L.n++;
                            }
                        }
                    }
                    nset = L.n;
                    if (nset > budget)
                        fits = 0;
                }
                /* Enough lanes to produce n texels, tpl each?  With edge
                 * remapping any ceil(n / tpl) active lanes do (producer of
                 * texel i is lane h(i mod na, A), in round i div na); without
                 * it, lanes 0..min(n, 32)-1 must all be active (producer of
                 * texel i is lane i mod 32). */
                if (fits) {
                    if (edge_remap) {
                        if (L.n > tpl * nactive) fits = 0;
                    } else {
                        int lanes = L.n < 32 ? L.n : 32;
                        uint32_t need = lanes >= 32 ? 0xffffffffu : ((1u << lanes) - 1u);
                        if ((A & need) != need) fits = 0;
                    }
                }
                path = fits ? PATH_SUCCESS : PATH_FALLBACK_BUDGET;
            }
            if (tile_path) tile_path[tile_id] = path;
            if (tile_n) tile_n[tile_id] = nset;

            if (!fits) {
                if (path == PATH_FALLBACK_MINIFIED) st.tiles_fallback_minified++;
                else st.tiles_fallback_budget++;
                if (path == PATH_FALLBACK_BUDGET && fallback) {
                    fallback_c(src, lane, A, fallback, view, seed, fp64, W, out, outd, evals, grouped ? &G : NULL);
                    continue;
                }
                for (int l = 0; l < 32; ++l) {
                    if (!lane[l].active) continue;
                    size_t idx = (size_t)lane[l].py * W + lane[l].px;
                    int tx, ty;
                    stf_lane(src, &lane[l], filter, view, seed, fp64, out, outd, evals, idx, &tx, &ty);
                    group_note(grouped ? &G : NULL, src, tx, ty);
                }
                continue;
            }
            st.tiles_success++;
            /* Step 2: texel i is produced once, by lane h(i mod na, A) (or lane
             * i mod 32); a lane produces up to tpl texels. */
            float valf[128][4];
            double vald[128][4];
            for (int i = 0; i < L.n; ++i) {
                int producer = edge_remap ? oracle_h(&A, 1, i % nactive) : i % 32;
                const pixel_setup *p = &lane[producer];
                size_t idx = (size_t)p->py * W + p->px;
                fetch_texel(src, L.x[i], L.y[i], valf[i], vald[i]);
                evals[idx]++;
                group_note(grouped ? &G : NULL, src, L.x[i], L.y[i]);
            }
            /* Step 3: every active lane gathers its F x F taps and filters. */
            for (int l = 0; l < 32; ++l) {
                if (!lane[l].active) continue;
                const pixel_setup *p = &lane[l];
                size_t idx = (size_t)p->py * W + p->px;
                float w[16], pv[16][4], o[4];
                double pd[16][4], od[4];
                const int nt = filter_weights(filter, p->s, p->t, w);
                for (int k = 0; k < nt; ++k) {
                    int j = list_find(&L, p->ulx - off + k % F, p->uly - off + k / F);
                    if (j < 0)
                        return -2; /* cannot happen: the set covers every tap */
                    for (int ch = 0; ch < 4; ++ch) {
                        pv[k][ch] = valf[j][ch];
                        pd[k][ch] = vald[j][ch];
                    }
                }
                filter_n(nt, w, pv, pd, fp64, o, od);
                for (int ch = 0; ch < 4; ++ch) {
                    if (out) out[4 * idx + ch] = o[ch];
                    if (outd) outd[4 * idx + ch] = od[ch];
                }
            }
        }
    }
    /* Total evaluations = sum of the per-pixel counts. */
    int64_t tot = 0;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x)
            tot += evals[(size_t)y * W + x];
    st.texel_evals = tot;
    unique += G.n;
    if (stats_out) {
        stats_out[0] = st.tiles_total;
        stats_out[1] = st.tiles_empty;
        stats_out[2] = st.tiles_direct;
        stats_out[3] = st.tiles_success;
        stats_out[4] = st.tiles_fallback_budget;
        stats_out[5] = st.tiles_fallback_minified;
        stats_out[6] = st.pixels_active;
        stats_out[7] = st.texel_evals;
        stats_out[8] = grouped ? unique : st.texel_evals;
    }
    return 0;
}

/* Exact block decode, FP32 arithmetic with the rounding described above. */
int oracle_filter(const uint8_t *blocks, int Wt, int Ht, const float *uv, const float *jac, const uint8_t *cov,
                  int W, int H, int view, int alg, uint64_t seed, int tile_w, int tile_h, int budget,
                  int mask_dim, int edge_remap, int group_tiles, int fallback, int tpl, int filter, int y0,
                  float *out, uint8_t *evals, int32_t *tile_path, int32_t *tile_n, int64_t *stats)
{
    if (Wt <= 0 || Ht <= 0 || Wt % 4 || Ht % 4 || !blocks)
        return -1;
    texel_source src = {0, Wt, Ht, blocks, NULL};
    return oracle_filter_ex(&src, uv, jac, cov, W, H, view, alg, seed, tile_w, tile_h, budget, mask_dim,
                            edge_remap, group_tiles, fallback, tpl, filter, y0, 0, out, NULL, evals, tile_path,
                            tile_n, stats);
}

/* Learned decode: texel values from the FP64 MLP, filter in double. */
int oracle_filter_learned_f64(const void *mlp, int Wt, int Ht, const float *uv, const float *jac,
                              const uint8_t *cov, int W, int H, int view, int alg, uint64_t seed, int tile_w,
                              int tile_h, int budget, int mask_dim, int edge_remap, int group_tiles,
                              int fallback, int tpl, int filter, int y0, double *outd, uint8_t *evals,
                              int32_t *tile_path, int32_t *tile_n, int64_t *stats)
{
    if (Wt <= 0 || Ht <= 0 || !mlp)
        return -1;
    texel_source src = {1, Wt, Ht, NULL, mlp};
    return oracle_filter_ex(&src, uv, jac, cov, W, H, view, alg, seed, tile_w, tile_h, budget, mask_dim,
                            edge_remap, group_tiles, fallback, tpl, filter, y0, 1, NULL, outd, evals, tile_path,
                            tile_n, stats);
}

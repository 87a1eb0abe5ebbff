/*
 * ctf_oracle_mlp.c -- FP64 oracle for the learned texel decode.
 *
 * TEST INFRASTRUCTURE ONLY (see ctf_oracle.c): loaded by tests/, smoke() and
 * bench.py's CPU-baseline leg, never by the product library.
 *
 * The paper evaluates texels with a neural decompressor (Sec. 4.3.1, NTC
 * "inference on sample") but defines no network; this file is the FP64 form of
 * the project's stand-in, written out as its plain definition:
 *
 *   feature f(x, y) = concat over grids g of the bilinear sample of latent
 *                     grid L_g at the texel centre, i.e. at grid position
 *                     ((x + 0.5) * Gw/Wt - 0.5, (y + 0.5) * Gh/Ht - 0.5),
 *                     taps clamped to the grid;
 *   h1 = relu(W1 f + b1), h2 = relu(W2 h1 + b2), y = W3 h2 + b3,
 *   texel value = saturate(y) (clamped to [0, 1]) when saturate is set.
 *
 * Parameters arrive as doubles: the caller dequantises the stored FP16 / FP8
 * weights and latents exactly (every FP16 and E4M3 value is a double).
 * Training loss (used for the gradient check): L = (1/B) sum_b sum_c
 * (y_bc - target_bc)^2 on the unsaturated output.
 */
#include <stdint.h>
#include <stddef.h>
#include <string.h>
#include <math.h>

typedef struct {
    int ch;                  /* channels per grid */
    int gw[2], gh[2];        /* grid sizes */
    const double *latent[2]; /* [gh][gw][ch], channel-last */
    int nin;                 /* = 2*ch */
    int hidden;
    int nout;
    const double *w1;        /* [hidden][nin] */
    const double *b1;        /* [hidden] */
    const double *w2;        /* [hidden][hidden] */
    const double *b2;
    const double *w3;        /* [nout][hidden] */
    const double *b3;
    int saturate;
} oracle_mlp;

#define MAXF 64
#define MAXH 256

typedef struct {
    int ix[2][4], iy[2][4]; /* clamped tap coordinates per grid */
    double w[2][4];         /* bilinear weights per grid */
} feature_taps;

static void feature_taps_of(const oracle_mlp *m, int Wt, int Ht, int x, int y, feature_taps *ft)
{
    for (int g = 0; g < 2; ++g) {
        double gx = ((double)x + 0.5) * ((double)m->gw[g] / (double)Wt) - 0.5;
        double gy = ((double)y + 0.5) * ((double)m->gh[g] / (double)Ht) - 0.5;
        double fx0 = floor(gx), fy0 = floor(gy);
        double fx = gx - fx0, fy = gy - fy0;
        int x0 = (int)fx0, y0 = (int)fy0;
        for (int k = 0; k < 4; ++k) {
            int tx = x0 + k % 2, ty = y0 + k / 2;
            if (tx < 0) tx = 0;
            if (tx > m->gw[g] - 1) tx = m->gw[g] - 1;
            if (ty < 0) ty = 0;
            if (ty > m->gh[g] - 1) ty = m->gh[g] - 1;
            ft->ix[g][k] = tx;
            ft->iy[g][k] = ty;
        }
        ft->w[g][0] = (1.0 - fx) * (1.0 - fy);
        ft->w[g][1] = fx * (1.0 - fy);
        ft->w[g][2] = (1.0 - fx) * fy;
        ft->w[g][3] = fx * fy;
    }
}

void oracle_mlp_features_f64(const void *mp, int Wt, int Ht, int x, int y, double *f)
{
    const oracle_mlp *m = (const oracle_mlp *)mp;
    feature_taps ft;
    feature_taps_of(m, Wt, Ht, x, y, &ft);
    for (int g = 0; g < 2; ++g) {
        for (int c = 0; c < m->ch; ++c) {
            double acc = 0.0;
            for (int k = 0; k < 4; ++k) {
                size_t off = ((size_t)ft.iy[g][k] * m->gw[g] + ft.ix[g][k]) * m->ch + c;
                acc += ft.w[g][k] * m->latent[g][off];
            }
            f[g * m->ch + c] = acc;
        }
    }
}

/* Forward pass of one feature vector; keeps the hidden activations. */
static void forward(const oracle_mlp *m, const double *f, double *h1, double *h2, double *y)
{
    for (int o = 0; o < m->hidden; ++o) {
        double acc = m->b1[o];
        for (int i = 0; i < m->nin; ++i)
            acc += m->w1[(size_t)o * m->nin + i] * f[i];
        h1[o] = acc > 0.0 ? acc : 0.0;
    }
    for (int o = 0; o < m->hidden; ++o) {
        double acc = m->b2[o];
        for (int i = 0; i < m->hidden; ++i)
            acc += m->w2[(size_t)o * m->hidden + i] * h1[i];
        h2[o] = acc > 0.0 ? acc : 0.0;
    }
    for (int o = 0; o < m->nout; ++o) {
        double acc = m->b3[o];
        for (int i = 0; i < m->hidden; ++i)
            acc += m->w3[(size_t)o * m->hidden + i] * h2[i];
        y[o] = acc;
    }
}

/* Texel value of the learned decode (x, y must already be inside the
 * texture; the filter clamps before calling). */
void oracle_mlp_texel_f64(const void *mp, int Wt, int Ht, int x, int y, double out[4])
{
    const oracle_mlp *m = (const oracle_mlp *)mp;
    double f[MAXF], h1[MAXH], h2[MAXH], yv[8];
    oracle_mlp_features_f64(m, Wt, Ht, x, y, f);
    forward(m, f, h1, h2, yv);
    for (int c = 0; c < 4; ++c) {
        double v = c < m->nout ? yv[c] : 1.0;
        if (m->saturate) v = v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v);
        out[c] = v;
    }
}

/* Batch decode of n texels (x[i], y[i]) to out[n][4]. */
void oracle_mlp_decode_f64(const void *mp, int Wt, int Ht, int n, const int32_t *xs, const int32_t *ys, double *out)
{
    for (int i = 0; i < n; ++i)
        oracle_mlp_texel_f64(mp, Wt, Ht, xs[i], ys[i], out + 4 * (size_t)i);
}

/*
 * Loss and gradients of L = (1/B) sum_b sum_c (y_bc - t_bc)^2 over a batch.
 * Gradient arrays have the shapes of the parameters and are overwritten;
 * dlat[g] has the shape of latent[g].  Any gradient pointer may be NULL.
 */
double oracle_mlp_loss_grad_f64(const void *mp, int Wt, int Ht, int B, const int32_t *xs, const int32_t *ys,
                                const double *targets, double *dw1, double *db1, double *dw2, double *db2,
                                double *dw3, double *db3, double *dlat0, double *dlat1)
{
    const oracle_mlp *m = (const oracle_mlp *)mp;
    int H = m->hidden, I = m->nin, O = m->nout;
    if (dw1) memset(dw1, 0, sizeof(double) * (size_t)H * I);
    if (db1) memset(db1, 0, sizeof(double) * (size_t)H);
    if (dw2) memset(dw2, 0, sizeof(double) * (size_t)H * H);
    if (db2) memset(db2, 0, sizeof(double) * (size_t)H);
    if (dw3) memset(dw3, 0, sizeof(double) * (size_t)O * H);
    if (db3) memset(db3, 0, sizeof(double) * (size_t)O);
    double *dlat[2] = {dlat0, dlat1};
    for (int g = 0; g < 2; ++g)
        if (dlat[g]) memset(dlat[g], 0, sizeof(double) * (size_t)m->gw[g] * m->gh[g] * m->ch);
    double loss = 0.0;
    for (int b = 0; b < B; ++b) {
        double f[MAXF], h1[MAXH], h2[MAXH], y[8];
        feature_taps ft;
        feature_taps_of(m, Wt, Ht, xs[b], ys[b], &ft);
        oracle_mlp_features_f64(m, Wt, Ht, xs[b], ys[b], f);
        forward(m, f, h1, h2, y);
        double dy[8], dh2[MAXH], dh1[MAXH], df[MAXF];
        for (int c = 0; c < O; ++c) {
            double e = y[c] - targets[(size_t)b * O + c];
            loss += e * e;
            dy[c] = 2.0 * e / (double)B;
        }
        /* layer 3 */
        for (int i = 0; i < H; ++i) dh2[i] = 0.0;
        for (int c = 0; c < O; ++c) {
            if (db3) db3[c] += dy[c];
            for (int i = 0; i < H; ++i) {
                if (dw3) dw3[(size_t)c * H + i] += dy[c] * h2[i];
                dh2[i] += dy[c] * m->w3[(size_t)c * H + i];
            }
        }
        for (int i = 0; i < H; ++i) if (!(h2[i] > 0.0)) dh2[i] = 0.0;
        /* layer 2 */
        for (int i = 0; i < H; ++i) dh1[i] = 0.0;
        for (int o = 0; o < H; ++o) {
            if (db2) db2[o] += dh2[o];
            for (int i = 0; i < H; ++i) {
                if (dw2) dw2[(size_t)o * H + i] += dh2[o] * h1[i];
                dh1[i] += dh2[o] * m->w2[(size_t)o * H + i];
            }
        }
        for (int i = 0; i < H; ++i) if (!(h1[i] > 0.0)) dh1[i] = 0.0;
        /* layer 1 */
        for (int i = 0; i < I; ++i) df[i] = 0.0;
        for (int o = 0; o < H; ++o) {
            if (db1) db1[o] += dh1[o];
            for (int i = 0; i < I; ++i) {
                if (dw1) dw1[(size_t)o * I + i] += dh1[o] * f[i];
                df[i] += dh1[o] * m->w1[(size_t)o * I + i];
            }
        }
        /* latent grids: each feature is a bilinear blend of 4 grid taps */
        for (int g = 0; g < 2; ++g) {
            if (!dlat[g]) continue;
            for (int k = 0; k < 4; ++k) {
                size_t base = ((size_t)ft.iy[g][k] * m->gw[g] + ft.ix[g][k]) * m->ch;
                for (int c = 0; c < m->ch; ++c)
                    dlat[g][base + c] += ft.w[g][k] * df[g * m->ch + c];
            }
        }
    }
    return loss / (double)B;
}

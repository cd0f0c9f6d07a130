/*
 * nlc_oracle.c -- plain, slow, scalar FP64 CPU oracle for the local
 * autoregressive image compressor of "Parallel Neural Local Lossless
 * Compression" (Zhang, Townsend, Kang, Barber).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the test-suite, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code, header, table or constant
 * generator with the CUDA library.
 *
 * What it computes, and where it comes from:
 *   - the local model of Eq. 3 (Section 2.1): pixel (i,j) is conditioned on
 *     rows i-h..i-1, columns j-h..j+h and on row i, columns j-h..j-1, with
 *     zero padding outside the coding unit;
 *   - the local PixelCNN of Section 2.1: a masked first layer whose receptive
 *     field is exactly that context, then 1x1 layers (residual blocks, ELU)
 *     and a 1x1 head;
 *   - a K-component discretized logistic mixture with channel-coupled RGB
 *     means as the per-pixel distribution (joint mixture, coded R, G|R,
 *     B|R,G by the chain rule);
 *   - the deterministic CDF -> 16-bit frequency quantiser;
 *   - a 32-bit rANS stream coder (ANS, Section 2), one stream per coding unit
 *     or per unit row;
 *   - sequential raster-order encode/decode (the sequential baseline of
 *     Section 4), which by Section 3 gives exactly the result that the
 *     wavefront schedule of Algorithm 1 must reproduce;
 *   - the mean negative log-likelihood in bits per dimension (Eq. 2) and its
 *     analytic gradient.
 * Everything is double precision; nothing is blocked, fused or reordered.
 */
#define _GNU_SOURCE
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_LN2
#define M_LN2 0.69314718055994530942
#endif

#define ORC_MQ 65280 /* 2^16 - 256: mass spread by the CDF, 1 count per symbol is reserved */

typedef struct {
    int h, C, R, K;
} orc_cfg;

static int n_ctx(int h) { return 2 * h * (h + 1); }      /* context pixels, Eq. 3 */
static int n_feat(int h) { return 3 * n_ctx(h); }        /* context features (RGB) */

long orc_num_weights(int h, int C, int R, int K)
{
    long F = n_feat(h);
    return (long)C * F + C + (long)R * 2 * ((long)C * C + C) + 10L * K * C + 10L * K;
}

/* Offsets of the tensors inside the flat weight vector (storage order:
 * W0[C][F], b0[C], then per residual block W1[C][C], b1[C], W2[C][C], b2[C],
 * then WH[10K][C], bH[10K]). */
typedef struct {
    const double *W0, *b0, *WH, *bH;
    const double *W1[16], *b1[16], *W2[16], *b2[16];
} orc_w;

static void split_weights(const orc_cfg *c, const double *w, orc_w *o)
{
    long F = n_feat(c->h), C = c->C;
    o->W0 = w; w += C * F;
    o->b0 = w; w += C;
    for (int r = 0; r < c->R; r++) {
        o->W1[r] = w; w += C * C;
        o->b1[r] = w; w += C;
        o->W2[r] = w; w += C * C;
        o->b2[r] = w; w += C;
    }
    o->WH = w; w += 10L * c->K * C;
    o->bH = w;
}

/* Gradient accumulator with the same layout. */
typedef struct {
    double *W0, *b0, *WH, *bH;
    double *W1[16], *b1[16], *W2[16], *b2[16];
} orc_g;

static void split_grad(const orc_cfg *c, double *w, orc_g *o)
{
    long F = n_feat(c->h), C = c->C;
    o->W0 = w; w += C * F;
    o->b0 = w; w += C;
    for (int r = 0; r < c->R; r++) {
        o->W1[r] = w; w += C * C;
        o->b1[r] = w; w += C;
        o->W2[r] = w; w += C * C;
        o->b2[r] = w; w += C;
    }
    o->WH = w; w += 10L * c->K * C;
    o->bH = w;
}

/* ------------------------------------------------------------------ */
/* Section 2.1, Eq. 3: the causal context of pixel (i, j) in a unit.   */
/* Position p enumerates the unmasked taps of a (2h+1)x(2h+1) kernel   */
/* in raster order: rows dy=-h..-1 with dx=-h..h, then dy=0, dx=-h..-1. */
/* Feature 3p+c is channel c of that pixel, scaled to (2v-255)/255;     */
/* taps outside the unit are 0 (zero padding).                          */
/* ------------------------------------------------------------------ */
static void gather_context(int h, const uint8_t *img, int img_W, int y0, int x0, int Hu,
                           int Wu, int i, int j, double *x)
{
    int p = 0;
    for (int dy = -h; dy <= 0; dy++) {
        int dx_end = (dy < 0) ? h : -1;
        for (int dx = -h; dx <= dx_end; dx++, p++) {
            int ii = i + dy, jj = j + dx;
            for (int c = 0; c < 3; c++) {
                double v = 0.0;
                if (ii >= 0 && ii < Hu && jj >= 0 && jj < Wu) {
                    int pv = img[((long)(y0 + ii) * img_W + (x0 + jj)) * 3 + c];
                    v = (2.0 * pv - 255.0) / 255.0;
                }
                x[3 * p + c] = v;
            }
        }
    }
}

static double elu(double x) { return x > 0 ? x : expm1(x); }
static double elu_d(double x) { return x > 0 ? 1.0 : exp(x); }

/* Activations of one forward pass, kept for the backward pass. */
typedef struct {
    double *x;      /* [F]             */
    double *a;      /* [(R+1)][C] residual stream a_0..a_R */
    double *hpre;   /* [R][C] pre-activation of the inner 1x1 layer */
    double *out;    /* [10K]           */
} orc_act;

/* Local PixelCNN forward (Section 2.1; Section 4 uses 1x1 ResNet blocks):
 *   a_0 = W0 x + b0
 *   a_{r+1} = a_r + W2_r ELU(W1_r ELU(a_r) + b1_r) + b2_r
 *   out = WH ELU(a_R) + bH                                           */
static void forward_px(const orc_cfg *c, const orc_w *W, orc_act *A)
{
    int C = c->C, F = n_feat(c->h), NO = 10 * c->K;
    double *a0 = A->a;
    for (int o = 0; o < C; o++) {
        double s = W->b0[o];
        for (int f = 0; f < F; f++) s += W->W0[(long)o * F + f] * A->x[f];
        a0[o] = s;
    }
    double *u = (double *)malloc(sizeof(double) * C);
    double *v = (double *)malloc(sizeof(double) * C);
    for (int r = 0; r < c->R; r++) {
        double *ar = A->a + (long)r * C, *an = A->a + (long)(r + 1) * C;
        double *hp = A->hpre + (long)r * C;
        for (int k = 0; k < C; k++) u[k] = elu(ar[k]);
        for (int o = 0; o < C; o++) {
            double s = W->b1[r][o];
            for (int k = 0; k < C; k++) s += W->W1[r][(long)o * C + k] * u[k];
            hp[o] = s;
        }
        for (int k = 0; k < C; k++) v[k] = elu(hp[k]);
        for (int o = 0; o < C; o++) {
            double s = W->b2[r][o];
            for (int k = 0; k < C; k++) s += W->W2[r][(long)o * C + k] * v[k];
            an[o] = ar[o] + s;
        }
    }
    double *aR = A->a + (long)c->R * C;
    for (int k = 0; k < C; k++) u[k] = elu(aR[k]);
    for (int o = 0; o < NO; o++) {
        double s = W->bH[o];
        for (int k = 0; k < C; k++) s += W->WH[(long)o * C + k] * u[k];
        A->out[o] = s;
    }
    free(u);
    free(v);
}

static void act_alloc(const orc_cfg *c, orc_act *A)
{
    A->x = (double *)calloc(n_feat(c->h), sizeof(double));
    A->a = (double *)calloc((size_t)(c->R + 1) * c->C, sizeof(double));
    A->hpre = (double *)calloc((size_t)(c->R > 0 ? c->R : 1) * c->C, sizeof(double));
    A->out = (double *)calloc(10 * c->K, sizeof(double));
}

static void act_free(orc_act *A)
{
    free(A->x); free(A->a); free(A->hpre); free(A->out);
}

/* ------------------------------------------------------------------ */
/* Discretized logistic mixture.                                        */
/* Bin v (0..255) of the scaled value x_v = (2v-255)/255 is the         */
/* interval [e_v, e_{v+1}) with e_b = (2b-256)/255, e_0 = -inf,         */
/* e_256 = +inf, so the 256 bin masses of a component sum to one.       */
/* ------------------------------------------------------------------ */
static double edge(int b) { return (2.0 * b - 256.0) / 255.0; }

double orc_sigmoid(double z) { return z >= 0 ? 1.0 / (1.0 + exp(-z)) : exp(z) / (1.0 + exp(z)); }
static double softplus(double z) { return z > 0 ? z + log1p(exp(-z)) : log1p(exp(z)); }
/* log(1 - e^{-d}) for d > 0, accurate for small and large d (Maechler, 2012). */
static double log1mexp(double d) { return d <= M_LN2 ? log(-expm1(-d)) : log1p(-exp(-d)); }

/* log P(v) for one logistic component with location m and log-scale ls.
 * With a = (e_{v+1}-m)/s and b = (e_v-m)/s:
 *   P = sigma(a) - sigma(b) = sigma(a) sigma(-b) (1 - e^{-(a-b)}),
 * so log P = -softplus(-a) - softplus(b) + log(1 - e^{-(a-b)}), where
 * a-b = (2/255)/s.  Edge bins: log sigma(a) and log(1-sigma(b)).       */
double orc_log_bin_mass(double m, double ls, int v)
{
    double inv = exp(-ls);
    if (v <= 0) return -softplus(-(edge(1) - m) * inv);
    if (v >= 255) return -softplus((edge(255) - m) * inv);
    double a = (edge(v + 1) - m) * inv;
    double b = (edge(v) - m) * inv;
    return -softplus(-a) - softplus(b) + log1mexp((2.0 / 255.0) * inv);
}

/* Mixture parameters of one pixel from the 10K network outputs:
 * [0,K) mixture logits; [K,4K) locations mu_c,k; [4K,7K) log-scales
 * (clamped below at -7); [7K,10K) raw coupling coefficients alpha, beta,
 * gamma (squashed by tanh).  Coupled locations in the scaled domain:
 *   m_R = mu_R, m_G = mu_G + alpha x_R, m_B = mu_B + beta x_R + gamma x_G. */
typedef struct {
    int K;
    double logpi[64];
    double m[3][64];
    double ls[3][64];
    double coef[3][64];
} orc_mix;

static void mix_from_params(int K, const double *p, int r, int g, orc_mix *M)
{
    M->K = K;
    double mx = p[0];
    for (int k = 1; k < K; k++) mx = p[k] > mx ? p[k] : mx;
    double s = 0;
    for (int k = 0; k < K; k++) s += exp(p[k] - mx);
    double lse = mx + log(s);
    double xr = (2.0 * r - 255.0) / 255.0, xg = (2.0 * g - 255.0) / 255.0;
    for (int k = 0; k < K; k++) {
        M->logpi[k] = p[k] - lse;
        for (int c = 0; c < 3; c++) {
            double l = p[4 * K + c * K + k];
            M->ls[c][k] = l < -7.0 ? -7.0 : l;
            M->coef[c][k] = tanh(p[7 * K + c * K + k]);
        }
        M->m[0][k] = p[K + k];
        M->m[1][k] = p[2 * K + k] + M->coef[0][k] * xr;
        M->m[2][k] = p[3 * K + k] + M->coef[1][k] * xr + M->coef[2][k] * xg;
    }
}

/* Component weights for coding channel ch given the already-coded channels:
 * R: pi_k; G: prop. to pi_k P_Rk(r); B: prop. to pi_k P_Rk(r) P_Gk(g)
 * (chain rule of the joint mixture). */
static void channel_weights(const orc_mix *M, int ch, int r, int g, double *w)
{
    int K = M->K;
    double lw[64], mx = -INFINITY;
    for (int k = 0; k < K; k++) {
        double l = M->logpi[k];
        if (ch >= 1) l += orc_log_bin_mass(M->m[0][k], M->ls[0][k], r);
        if (ch >= 2) l += orc_log_bin_mass(M->m[1][k], M->ls[1][k], g);
        lw[k] = l;
        if (l > mx) mx = l;
    }
    double s = 0;
    for (int k = 0; k < K; k++) { w[k] = exp(lw[k] - mx); s += w[k]; }
    for (int k = 0; k < K; k++) w[k] /= s;
}

/* CDF -> integer frequencies.  F(b) = sum_k w_k sigma((e_b - m_k)/s_k) for
 * the boundaries b = 1..255; q_b = clamp(rint(65280 F(b)), 0, 65280) with
 * round-half-to-even; Q_b = max(Q_{b-1}, q_b), Q_0 = 0; cum_b = Q_b + b,
 * cum_256 = 2^16.  Then freq_v = cum_{v+1} - cum_v >= 1 and the
 * frequencies sum to 2^16. */
void orc_quantise_cdf(const double *F, uint32_t *cum)
{
    long Q = 0;
    cum[0] = 0;
    for (int b = 1; b <= 255; b++) {
        double q = nearbyint((double)ORC_MQ * F[b]);
        if (q < 0) q = 0;
        if (q > ORC_MQ) q = ORC_MQ;
        if ((long)q > Q) Q = (long)q;
        cum[b] = (uint32_t)(Q + b);
    }
    cum[256] = 65536u;
}

static void channel_table(const orc_mix *M, int ch, int r, int g, uint32_t *cum)
{
    double w[64], F[257];
    channel_weights(M, ch, r, g, w);
    F[0] = 0.0;
    F[256] = 1.0;
    for (int b = 1; b <= 255; b++) {
        double s = 0;
        for (int k = 0; k < M->K; k++)
            s += w[k] * orc_sigmoid((edge(b) - M->m[ch][k]) * exp(-M->ls[ch][k]));
        F[b] = s;
    }
    orc_quantise_cdf(F, cum);
}

/* Tables of the three channels of one pixel (cum[3][257]) from its network
 * outputs and its R and G values (needed for G's and B's tables). */
void orc_pixel_tables(int K, const double *params, int r, int g, uint32_t *cum)
{
    orc_mix M;
    mix_from_params(K, params, r, g, &M);
    for (int ch = 0; ch < 3; ch++) channel_table(&M, ch, r, g, cum + 257 * ch);
}

/* Model code length of one pixel, -log2 p(r,g,b), with
 * p = sum_k pi_k P_Rk(r) P_Gk(g|r) P_Bk(b|r,g). */
double orc_pixel_bits(int K, const double *params, int r, int g, int b)
{
    orc_mix M;
    mix_from_params(K, params, r, g, &M);
    double l[64], mx = -INFINITY;
    for (int k = 0; k < K; k++) {
        l[k] = M.logpi[k] + orc_log_bin_mass(M.m[0][k], M.ls[0][k], r) +
               orc_log_bin_mass(M.m[1][k], M.ls[1][k], g) +
               orc_log_bin_mass(M.m[2][k], M.ls[2][k], b);
        if (l[k] > mx) mx = l[k];
    }
    double s = 0;
    for (int k = 0; k < K; k++) s += exp(l[k] - mx);
    return -(mx + log(s)) / M_LN2;
}

/* Probability of channel value v under channel ch's coding distribution,
 * given (r, g): sum_k w_k P_k(v) with the chain-rule weights above. */
double orc_channel_prob(int K, const double *params, int ch, int r, int g, int v)
{
    orc_mix M;
    double w[64], s = 0;
    mix_from_params(K, params, r, g, &M);
    channel_weights(&M, ch, r, g, w);
    for (int k = 0; k < K; k++) s += w[k] * exp(orc_log_bin_mass(M.m[ch][k], M.ls[ch][k], v));
    return s;
}

/* ------------------------------------------------------------------ */
/* Network outputs of every pixel of an image under a unit partition.  */
/* patch = 0: one unit (the whole image); else P x P units in raster    */
/* order, ragged at the right and bottom edges.                         */
/* ------------------------------------------------------------------ */
static void unit_of(int H, int W, int patch, int u, int *y0, int *x0, int *Hu, int *Wu)
{
    if (patch <= 0) { *y0 = 0; *x0 = 0; *Hu = H; *Wu = W; return; }
    int nx = (W + patch - 1) / patch;
    int py = u / nx, px = u % nx;
    *y0 = py * patch; *x0 = px * patch;
    *Hu = (H - *y0) < patch ? (H - *y0) : patch;
    *Wu = (W - *x0) < patch ? (W - *x0) : patch;
}

int orc_num_units(int H, int W, int patch)
{
    if (patch <= 0) return 1;
    return ((H + patch - 1) / patch) * ((W + patch - 1) / patch);
}

/* out: [H][W][10K] network outputs for every pixel. */
void orc_forward_image(int h, int C, int R, int K, const double *w, const uint8_t *img, int H,
                       int W, int patch, double *out)
{
    orc_cfg cfg = {h, C, R, K};
    orc_w Wt;
    orc_act A;
    split_weights(&cfg, w, &Wt);
    act_alloc(&cfg, &A);
    int nu = orc_num_units(H, W, patch), NO = 10 * K;
    for (int u = 0; u < nu; u++) {
        int y0, x0, Hu, Wu;
        unit_of(H, W, patch, u, &y0, &x0, &Hu, &Wu);
        for (int i = 0; i < Hu; i++)
            for (int j = 0; j < Wu; j++) {
                gather_context(h, img, W, y0, x0, Hu, Wu, i, j, A.x);
                forward_px(&cfg, &Wt, &A);
                memcpy(out + ((long)(y0 + i) * W + (x0 + j)) * NO, A.out, sizeof(double) * NO);
            }
    }
    act_free(&A);
}

/* Network outputs of a list of pixels (ys[n], xs[n]) of one image. */
void orc_forward_pixels(int h, int C, int R, int K, const double *w, const uint8_t *img, int H,
                        int W, int patch, int n, const int *ys, const int *xs, double *out)
{
    orc_cfg cfg = {h, C, R, K};
    orc_w Wt;
    orc_act A;
    split_weights(&cfg, w, &Wt);
    act_alloc(&cfg, &A);
    int NO = 10 * K;
    int nx = patch > 0 ? (W + patch - 1) / patch : 1;
    for (int q = 0; q < n; q++) {
        int y0, x0, Hu, Wu;
        int u = patch > 0 ? (ys[q] / patch) * nx + xs[q] / patch : 0;
        unit_of(H, W, patch, u, &y0, &x0, &Hu, &Wu);
        gather_context(h, img, W, y0, x0, Hu, Wu, ys[q] - y0, xs[q] - x0, A.x);
        forward_px(&cfg, &Wt, &A);
        memcpy(out + (long)q * NO, A.out, sizeof(double) * NO);
    }
    act_free(&A);
}

/* Model code length -log2 p(x_ij) of every pixel of an image under a unit
 * partition (bits[H][W]): the network outputs of orc_forward_image followed
 * by orc_pixel_bits, one pixel at a time. */
void orc_image_bits(int h, int C, int R, int K, const double *w, const uint8_t *img, int H, int W,
                    int patch, double *bits)
{
    orc_cfg cfg = {h, C, R, K};
    orc_w Wt;
    orc_act A;
    split_weights(&cfg, w, &Wt);
    act_alloc(&cfg, &A);
    int nu = orc_num_units(H, W, patch);
    for (int u = 0; u < nu; u++) {
        int y0, x0, Hu, Wu;
        unit_of(H, W, patch, u, &y0, &x0, &Hu, &Wu);
        for (int i = 0; i < Hu; i++)
            for (int j = 0; j < Wu; j++) {
                const uint8_t *px = img + ((long)(y0 + i) * W + (x0 + j)) * 3;
                gather_context(h, img, W, y0, x0, Hu, Wu, i, j, A.x);
                forward_px(&cfg, &Wt, &A);
                bits[(long)(y0 + i) * W + (x0 + j)] = orc_pixel_bits(K, A.out, px[0], px[1], px[2]);
            }
    }
    act_free(&A);
}

/* ------------------------------------------------------------------ */
/* 32-bit rANS (ANS, Section 2) with byte-wise renormalisation: state x  */
/* in [2^23, 2^31), 16-bit probability scale (M = 2^16), initial encoder */
/* state 2^23.  Encode of (start, freq): while x >= freq * 2^15 emit the  */
/* low byte and shift right by 8; then x = (x / freq) * 2^16 + x mod freq */
/* + start.  Symbols are encoded in reverse so that they decode forwards. */
/* Stream layout, in decoder read order: the final encoder state as four  */
/* bytes (most significant first), then the emitted bytes in reverse      */
/* emission order.  Decode: slot = x mod 2^16, s = the symbol with        */
/* cum_s <= slot < cum_{s+1}, x = freq_s (x >> 16) + slot - cum_s, then   */
/* while x < 2^23 shift a byte in.  A complete stream ends in state 2^23  */
/* with every byte consumed.                                              */
/* ------------------------------------------------------------------ */
#define ORC_RANS_L (1u << 23)

/* Returns the stream length in bytes, or -1 when cap is too small. */
long orc_rans_encode(long nsym, const uint32_t *start, const uint32_t *freq, uint8_t *out,
                     long cap)
{
    uint8_t *tmp = (uint8_t *)malloc((size_t)(2 * nsym + 4));
    long ne = 0;
    uint32_t x = ORC_RANS_L;
    for (long k = nsym - 1; k >= 0; k--) {
        uint32_t f = freq[k];
        uint32_t xmax = (ORC_RANS_L >> 16 << 8) * f;
        while (x >= xmax) {
            tmp[ne++] = (uint8_t)(x & 0xFFu);
            x >>= 8;
        }
        x = ((x / f) << 16) + (x % f) + start[k];
    }
    long n = ne + 4;
    if (n > cap) { free(tmp); return -1; }
    out[0] = (uint8_t)(x >> 24);
    out[1] = (uint8_t)(x >> 16);
    out[2] = (uint8_t)(x >> 8);
    out[3] = (uint8_t)x;
    for (long q = 0; q < ne; q++) out[4 + q] = tmp[ne - 1 - q];
    free(tmp);
    return n;
}

/* Decoder of one stream. */
typedef struct {
    uint32_t x;
    long pos, n;
    const uint8_t *w;
    int err;
} orc_rans_dec;

static void rans_dec_init(orc_rans_dec *d, const uint8_t *w, long n)
{
    d->w = w; d->n = n; d->err = 0;
    if (n < 4) { d->err = 1; d->x = 0; d->pos = n; return; }
    d->x = ((uint32_t)w[0] << 24) | ((uint32_t)w[1] << 16) | ((uint32_t)w[2] << 8) | w[3];
    d->pos = 4;
}

/* Decode one symbol with the cumulative table cum[0..256]. */
static int rans_dec_sym(orc_rans_dec *d, const uint32_t *cum)
{
    uint32_t slot = d->x & 0xFFFFu;
    int s = 0;
    while (s < 255 && cum[s + 1] <= slot) s++;
    uint32_t f = cum[s + 1] - cum[s];
    d->x = f * (d->x >> 16) + slot - cum[s];
    while (d->x < ORC_RANS_L) {
        if (d->pos < d->n) d->x = (d->x << 8) | d->w[d->pos++];
        else { d->err = 1; break; }
    }
    return s;
}

static int rans_dec_done(const orc_rans_dec *d)
{
    return !d->err && d->x == ORC_RANS_L && d->pos == d->n;
}

/* Decode nsym symbols with given per-symbol tables cum[nsym][257].
 * Returns 0 on success (final state 2^23, every byte consumed). */
int orc_rans_decode(const uint8_t *w, long n, long nsym, const uint32_t *cum, int32_t *sym)
{
    orc_rans_dec d;
    rans_dec_init(&d, w, n);
    for (long k = 0; k < nsym; k++) sym[k] = rans_dec_sym(&d, cum + 257 * k);
    return rans_dec_done(&d) ? 0 : 1;
}

/* ------------------------------------------------------------------ */
/* Image codec in raster order (sequential decode of Section 4).        */
/* Streams: layout 0 = one per unit (raster over the unit's pixels),    */
/* layout 1 = one per unit row (its pixels left to right).  Each pixel  */
/* contributes R, G, B in that order.  Stream order: units in raster    */
/* order, then rows.                                                     */
/* ------------------------------------------------------------------ */
int orc_num_streams(int H, int W, int patch, int layout)
{
    int nu = orc_num_units(H, W, patch);
    if (layout == 0) return nu;
    int n = 0;
    for (int u = 0; u < nu; u++) {
        int y0, x0, Hu, Wu;
        unit_of(H, W, patch, u, &y0, &x0, &Hu, &Wu);
        n += Hu;
    }
    return n;
}

/* Encode.  words: concatenated byte streams; lens[n_streams] bytes each.
 * bits_model (optional): sum over pixels of -log2 p.  bits_quant: sum of
 * -log2(freq/2^16) over the coded symbols.  Returns total bytes or -1.    */
long orc_encode_image(int h, int C, int R, int K, const double *w, const uint8_t *img, int H,
                      int W, int patch, int layout, uint8_t *words, long cap, int32_t *lens,
                      double *bits_model, double *bits_quant)
{
    orc_cfg cfg = {h, C, R, K};
    orc_w Wt;
    orc_act A;
    split_weights(&cfg, w, &Wt);
    act_alloc(&cfg, &A);
    int nu = orc_num_units(H, W, patch);
    long total = 0;
    int si = 0;
    double bm = 0, bq = 0;
    uint32_t cum[3 * 257];
    for (int u = 0; u < nu; u++) {
        int y0, x0, Hu, Wu;
        unit_of(H, W, patch, u, &y0, &x0, &Hu, &Wu);
        int nrows = layout == 0 ? 1 : Hu;
        long per = layout == 0 ? 3L * Hu * Wu : 3L * Wu;
        uint32_t *st = (uint32_t *)malloc(sizeof(uint32_t) * per);
        uint32_t *fr = (uint32_t *)malloc(sizeof(uint32_t) * per);
        for (int sr = 0; sr < nrows; sr++) {
            long k = 0;
            int i_lo = layout == 0 ? 0 : sr, i_hi = layout == 0 ? Hu : sr + 1;
            for (int i = i_lo; i < i_hi; i++)
                for (int j = 0; j < Wu; j++) {
                    const uint8_t *px = img + ((long)(y0 + i) * W + (x0 + j)) * 3;
                    gather_context(h, img, W, y0, x0, Hu, Wu, i, j, A.x);
                    forward_px(&cfg, &Wt, &A);
                    orc_pixel_tables(K, A.out, px[0], px[1], cum);
                    if (bits_model) bm += orc_pixel_bits(K, A.out, px[0], px[1], px[2]);
                    for (int c = 0; c < 3; c++) {
                        st[k] = cum[257 * c + px[c]];
                        fr[k] = cum[257 * c + px[c] + 1] - cum[257 * c + px[c]];
                        bq += -log2((double)fr[k] / 65536.0);
                        k++;
                    }
                }
            long n = orc_rans_encode(k, st, fr, words + total, cap - total);
            if (n < 0) { free(st); free(fr); act_free(&A); return -1; }
            lens[si++] = (int32_t)n;
            total += n;
        }
        free(st);
        free(fr);
    }
    act_free(&A);
    if (bits_model) *bits_model = bm;
    if (bits_quant) *bits_quant = bq;
    return total;
}

/* Decode in raster order over each unit.  Returns 0 on success. */
int orc_decode_image(int h, int C, int R, int K, const double *w, const uint8_t *words,
                     const int32_t *lens, int H, int W, int patch, int layout, uint8_t *img)
{
    orc_cfg cfg = {h, C, R, K};
    orc_w Wt;
    orc_act A;
    split_weights(&cfg, w, &Wt);
    act_alloc(&cfg, &A);
    memset(img, 0, (size_t)H * W * 3);
    int nu = orc_num_units(H, W, patch), bad = 0;
    long off = 0;
    int si = 0;
    uint32_t cum[257];
    for (int u = 0; u < nu; u++) {
        int y0, x0, Hu, Wu;
        unit_of(H, W, patch, u, &y0, &x0, &Hu, &Wu);
        orc_rans_dec d;
        if (layout == 0) { rans_dec_init(&d, words + off, lens[si]); off += lens[si++]; }
        for (int i = 0; i < Hu; i++) {
            if (layout == 1) { rans_dec_init(&d, words + off, lens[si]); off += lens[si++]; }
            for (int j = 0; j < Wu; j++) {
                uint8_t *px = img + ((long)(y0 + i) * W + (x0 + j)) * 3;
                orc_mix M;
                gather_context(h, img, W, y0, x0, Hu, Wu, i, j, A.x);
                forward_px(&cfg, &Wt, &A);
                mix_from_params(K, A.out, 0, 0, &M);
                channel_table(&M, 0, 0, 0, cum);
                int r = rans_dec_sym(&d, cum);
                mix_from_params(K, A.out, r, 0, &M);
                channel_table(&M, 1, r, 0, cum);
                int g = rans_dec_sym(&d, cum);
                mix_from_params(K, A.out, r, g, &M);
                channel_table(&M, 2, r, g, cum);
                int b = rans_dec_sym(&d, cum);
                px[0] = (uint8_t)r; px[1] = (uint8_t)g; px[2] = (uint8_t)b;
            }
            if (layout == 1) bad |= !rans_dec_done(&d);
        }
        if (layout == 0) bad |= !rans_dec_done(&d);
    }
    act_free(&A);
    return bad;
}

/* ------------------------------------------------------------------ */
/* Sampling from the model (Section 5 names sampling as another use of  */
/* the parallel schedules).  Counter-based uniforms: output k of the     */
/* SplitMix64 generator (Steele, Lea and Flood, 2014) seeded with s is    */
/* the finaliser applied to s + (k+1) gamma, gamma = 0x9E3779B97F4A7C15:  */
/*   z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27;                 */
/*   z *= 0x94D049BB133111EB; z ^= z >> 31.                               */
/* ------------------------------------------------------------------ */
uint64_t orc_splitmix64(uint64_t seed, uint64_t k)
{
    uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Uniform 16-bit value of channel c of pixel (y, x) of image n. */
uint32_t orc_sample_u16(uint64_t seed, int n, int y, int x, int c)
{
    uint64_t k = (((uint64_t)n << 21) + (uint64_t)y) << 21;
    k = (k + (uint64_t)x) * 3 + (uint64_t)c;
    return (uint32_t)(orc_splitmix64(seed, k) >> 48);
}

/* The symbol v with cum[v] <= u < cum[v+1] (inverse CDF of the table). */
static int table_symbol(const uint32_t *cum, uint32_t u)
{
    int v = 0;
    while (v < 255 && cum[v + 1] <= u) v++;
    return v;
}

/* Draws image n of a batch in raster order over each unit: every channel
 * is sampled from its quantised coding table with the uniform of
 * orc_sample_u16. */
void orc_sample_image(int h, int C, int R, int K, const double *w, int H, int W, int patch,
                      uint64_t seed, int n, uint8_t *img)
{
    orc_cfg cfg = {h, C, R, K};
    orc_w Wt;
    orc_act A;
    split_weights(&cfg, w, &Wt);
    act_alloc(&cfg, &A);
    memset(img, 0, (size_t)H * W * 3);
    int nu = orc_num_units(H, W, patch);
    uint32_t cum[257];
    for (int u = 0; u < nu; u++) {
        int y0, x0, Hu, Wu;
        unit_of(H, W, patch, u, &y0, &x0, &Hu, &Wu);
        for (int i = 0; i < Hu; i++)
            for (int j = 0; j < Wu; j++) {
                int y = y0 + i, x = x0 + j;
                uint8_t *px = img + ((long)y * W + x) * 3;
                orc_mix M;
                gather_context(h, img, W, y0, x0, Hu, Wu, i, j, A.x);
                forward_px(&cfg, &Wt, &A);
                mix_from_params(K, A.out, 0, 0, &M);
                channel_table(&M, 0, 0, 0, cum);
                int r = table_symbol(cum, orc_sample_u16(seed, n, y, x, 0));
                mix_from_params(K, A.out, r, 0, &M);
                channel_table(&M, 1, r, 0, cum);
                int g = table_symbol(cum, orc_sample_u16(seed, n, y, x, 1));
                mix_from_params(K, A.out, r, g, &M);
                channel_table(&M, 2, r, g, cum);
                int b = table_symbol(cum, orc_sample_u16(seed, n, y, x, 2));
                px[0] = (uint8_t)r; px[1] = (uint8_t)g; px[2] = (uint8_t)b;
            }
    }
    act_free(&A);
}

/* ------------------------------------------------------------------ */
/* Training objective (Eq. 2) in bits per dimension and its gradient.   */
/* loss = (1 / (3 N H W)) sum_pixels -log2 p(pixel); each image is one  */
/* unit (crops).                                                        */
/* ------------------------------------------------------------------ */

/* d(-ln p)/d(params) for one pixel, written to dp[10K]. */
static double pixel_nll_grad(int K, const double *p, int r, int g, int b, double *dp)
{
    orc_mix M;
    mix_from_params(K, p, r, g, &M);
    int v[3] = {r, g, b};
    double l[64], mx = -INFINITY;
    double dlm[3][64], dll[3][64]; /* d logP_ck / d m, d logP_ck / d ls */
    for (int k = 0; k < K; k++) {
        l[k] = M.logpi[k];
        for (int c = 0; c < 3; c++) {
            double m = M.m[c][k], ls = M.ls[c][k], inv = exp(-ls);
            l[k] += orc_log_bin_mass(m, ls, v[c]);
            if (v[c] == 0) {
                double a = (edge(1) - m) * inv, sa = orc_sigmoid(-a);
                dlm[c][k] = -inv * sa;
                dll[c][k] = -a * sa;
            } else if (v[c] == 255) {
                double bb = (edge(255) - m) * inv, sb = orc_sigmoid(bb);
                dlm[c][k] = inv * sb;
                dll[c][k] = bb * sb;
            } else {
                double a = (edge(v[c] + 1) - m) * inv, bb = (edge(v[c]) - m) * inv;
                double d = (2.0 / 255.0) * inv, gk = 1.0 / expm1(d);
                double sa = orc_sigmoid(-a), sb = orc_sigmoid(bb);
                dlm[c][k] = -inv * (sa - sb);
                dll[c][k] = -a * sa + bb * sb - gk * d;
            }
        }
        if (l[k] > mx) mx = l[k];
    }
    double s = 0, rho[64];
    for (int k = 0; k < K; k++) s += exp(l[k] - mx);
    double nll = -(mx + log(s));
    for (int k = 0; k < K; k++) rho[k] = exp(l[k] - mx) / s;
    double xr = (2.0 * r - 255.0) / 255.0, xg = (2.0 * g - 255.0) / 255.0;
    for (int k = 0; k < K; k++) {
        dp[k] = -rho[k] + exp(M.logpi[k]);
        double dmR = -rho[k] * dlm[0][k], dmG = -rho[k] * dlm[1][k], dmB = -rho[k] * dlm[2][k];
        dp[K + k] = dmR;
        dp[2 * K + k] = dmG;
        dp[3 * K + k] = dmB;
        for (int c = 0; c < 3; c++) {
            double raw = p[4 * K + c * K + k];
            dp[4 * K + c * K + k] = raw > -7.0 ? -rho[k] * dll[c][k] : 0.0;
        }
        double al = M.coef[0][k], be = M.coef[1][k], ga = M.coef[2][k];
        dp[7 * K + k] = dmG * xr * (1.0 - al * al);
        dp[8 * K + k] = dmB * xr * (1.0 - be * be);
        dp[9 * K + k] = dmB * xg * (1.0 - ga * ga);
    }
    return nll;
}

/* Mean bits per dimension over a batch of N HxW images, and (if grad is
 * not NULL) its gradient with respect to every weight (same layout). */
double orc_nll_grad(int h, int C, int R, int K, const double *w, const uint8_t *imgs, int N,
                    int H, int W, double *grad)
{
    orc_cfg cfg = {h, C, R, K};
    orc_w Wt;
    orc_g G;
    memset(&G, 0, sizeof G);
    orc_act A;
    split_weights(&cfg, w, &Wt);
    long nw = orc_num_weights(h, C, R, K);
    if (grad) { memset(grad, 0, sizeof(double) * nw); split_grad(&cfg, grad, &G); }
    act_alloc(&cfg, &A);
    int F = n_feat(h), NO = 10 * K;
    double *dp = (double *)malloc(sizeof(double) * NO);
    double *du = (double *)malloc(sizeof(double) * C);
    double *da = (double *)malloc(sizeof(double) * C);
    double *dh = (double *)malloc(sizeof(double) * C);
    double *t = (double *)malloc(sizeof(double) * C);
    double scale = 1.0 / (M_LN2 * 3.0 * (double)N * H * W);
    double total = 0;
    for (int n = 0; n < N; n++) {
        const uint8_t *img = imgs + (long)n * H * W * 3;
        for (int i = 0; i < H; i++)
            for (int j = 0; j < W; j++) {
                const uint8_t *px = img + ((long)i * W + j) * 3;
                gather_context(h, img, W, 0, 0, H, W, i, j, A.x);
                forward_px(&cfg, &Wt, &A);
                total += pixel_nll_grad(K, A.out, px[0], px[1], px[2], dp);
                if (!grad) continue;
                for (int o = 0; o < NO; o++) dp[o] *= scale;
                /* head */
                double *aR = A.a + (long)R * C;
                for (int k = 0; k < C; k++) du[k] = 0;
                for (int o = 0; o < NO; o++) {
                    G.bH[o] += dp[o];
                    for (int k = 0; k < C; k++) {
                        G.WH[(long)o * C + k] += dp[o] * elu(aR[k]);
                        du[k] += Wt.WH[(long)o * C + k] * dp[o];
                    }
                }
                for (int k = 0; k < C; k++) da[k] = du[k] * elu_d(aR[k]);
                /* residual blocks, last to first */
                for (int r = R - 1; r >= 0; r--) {
                    double *ar = A.a + (long)r * C, *hp = A.hpre + (long)r * C;
                    for (int k = 0; k < C; k++) t[k] = 0;
                    for (int o = 0; o < C; o++) {
                        G.b2[r][o] += da[o];
                        for (int k = 0; k < C; k++) {
                            G.W2[r][(long)o * C + k] += da[o] * elu(hp[k]);
                            t[k] += Wt.W2[r][(long)o * C + k] * da[o];
                        }
                    }
                    for (int k = 0; k < C; k++) dh[k] = t[k] * elu_d(hp[k]);
                    for (int k = 0; k < C; k++) t[k] = 0;
                    for (int o = 0; o < C; o++) {
                        G.b1[r][o] += dh[o];
                        for (int k = 0; k < C; k++) {
                            G.W1[r][(long)o * C + k] += dh[o] * elu(ar[k]);
                            t[k] += Wt.W1[r][(long)o * C + k] * dh[o];
                        }
                    }
                    for (int k = 0; k < C; k++) da[k] += t[k] * elu_d(ar[k]);
                }
                /* first layer */
                for (int o = 0; o < C; o++) {
                    G.b0[o] += da[o];
                    for (int f = 0; f < F; f++) G.W0[(long)o * F + f] += da[o] * A.x[f];
                }
            }
    }
    free(dp); free(du); free(da); free(dh); free(t);
    act_free(&A);
    return total / (M_LN2 * 3.0 * (double)N * H * W);
}

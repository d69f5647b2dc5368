/*
 * oracle.c -- plain FP64 CPU oracle of the CVC contourlet codec hot path.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).  Plain loops, no blocking, no
 * fusion, no reordering beyond what the definitions below state, so that a
 * reader can check each function against the paper by eye.
 *
 * Paper: S. Katsigiannis, G. Papaioannou, D. Maroulis, "CVC: The Contourlet
 * Video Compression algorithm for real-time applications", arXiv:1510.00561.
 * Section references (§) are to that paper.
 *
 * Readings taken where the paper is silent (each one is also listed in the
 * design notes of the repository):
 *   - colour: the integer lifting form YCoCg-R of Table 1 (Eq. 1-6);
 *   - chroma factor N = 4 (§4.1) read as 2x2 (4:2:0) area subsampling with
 *     a rounded box average; decoder upsampling = bilinear (§3.1) with
 *     centred sample siting, weights (9,3,3,1)/16;
 *   - LP (§2.1) with the CDF 9/7 pair [18], periodic extension, synthesis by
 *     the dual-frame rule x = d + G(c - H d);
 *   - DFB (§2.1): iterated two-channel fan filter banks in ladder (lifting)
 *     form with the 4-tap half-band (-1,9,9,-1)/16 prototype, resampled
 *     (sheared) coordinates from the third stage on, wedge-ordered tree;
 *   - lowpass normalisation (§3.4) = exact scale by 2^-L;
 *   - quantisation and rounding (§3.5, §3.6) = round half away from zero of
 *     c / QP, decided in single precision, int16 codes;
 *   - K/P differencing (§3.7) in wrapping 16-bit arithmetic, zero motion;
 *   - RLE (§3.8): per row, a non-zero value is one token, a maximal zero
 *     run of length n is the token pair (0, n).
 */
#include "oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <zlib.h>

static int wrapi(long a, int n) {
    long r = a % n;
    return (int)(r < 0 ? r + n : r);
}
static long floordiv(long a, long b) { /* b > 0 */
    long q = a / b;
    if ((a % b) != 0 && a < 0) q -= 1;
    return q;
}

/* ------------------------------------------------------------------ layout
 * Coefficient layout of one plane (§3.3: the coarsest lowpass image plus the
 * directional subbands of every scale): lowpass first, then levels 1 (finest)
 * to L, each level's 2^k subbands in tree order.  Plane sizes must be
 * multiples of the modulus so that every level and every DFB stage splits
 * evenly.                                                                   */
int or_modulus(int L, const int* k) {
    int m = 1 << L;
    for (int j = 1; j <= L; j++) {
        int kj = k[j - 1];
        int need = (1 << (j - 1)) * (kj >= 2 ? (1 << (kj - 1)) : 2);
        if (need > m) m = need;
    }
    return m;
}

int or_layout_make(int H, int W, int L, const int* k, or_layout* out) {
    if (L < 1 || L > OR_MAX_LEVELS || H <= 0 || W <= 0) return OR_EINVAL;
    for (int j = 0; j < L; j++)
        if (k[j] < 0 || k[j] > OR_MAX_K) return OR_EINVAL;
    int M = or_modulus(L, k);
    if (H % M || W % M) return OR_EINVAL;
    memset(out, 0, sizeof(*out));
    out->H = H; out->W = W; out->L = L;
    for (int j = 0; j < L; j++) out->k[j] = k[j];
    long off = 0;
    or_subband* s = &out->sb[0];
    s->off = 0; s->h = H >> L; s->w = W >> L; s->level = 0; s->dir = 0; s->kind = 0;
    off += (long)s->h * s->w;
    int n = 1;
    for (int j = 1; j <= L; j++) {
        int Hj = H >> (j - 1), Wj = W >> (j - 1), kj = k[j - 1];
        int nd = 1 << kj;
        for (int d = 0; d < nd; d++) {
            s = &out->sb[n++];
            s->off = off; s->level = j; s->dir = d;
            if (kj == 0) { s->h = Hj; s->w = Wj; s->kind = 3; }
            else if (kj == 1) { s->h = Hj; s->w = Wj / 2; s->kind = 4; }
            else if (d < nd / 2) { s->h = Hj >> (kj - 1); s->w = Wj / 2; s->kind = 1; }
            else { s->h = Hj / 2; s->w = Wj >> (kj - 1); s->kind = 2; }
            off += (long)s->h * s->w;
        }
    }
    out->nsub = n;
    out->total = off;
    return OR_OK;
}

/* ------------------------------------------------------------- CDF 9/7
 * §2.1 cites the Cohen-Daubechies 9-7 filters [18].  They are the
 * biorthogonal spline-variant pair obtained by splitting Daubechies'
 * polynomial P(y) = 1 + 4y + 10y^2 + 20y^3 (y = sin^2(w/2)): the real root
 * y0 goes to the 7-tap synthesis lowpass, the complex pair to the 9-tap
 * analysis lowpass, each with four zeros at w = pi and DC gain sqrt(2):
 *   H(w) = sqrt2 (1-y)^2 q(y),  G(w) = sqrt2 (1-y)^2 (1 - y/y0),
 *   q(y) = P(y) / (1 - y/y0).
 * Taps are computed by multiplying Laurent polynomials in z, with
 * 1 - y = (z + 2 + 1/z)/4 and y = (-z + 2 - 1/z)/4.                        */
static void lpoly_mul(const double* a, int ra, const double* b, int rb, double* out) {
    /* a has taps -ra..ra at a[0..2ra]; out has taps -(ra+rb)..(ra+rb) */
    int ro = ra + rb;
    for (int i = 0; i <= 2 * ro; i++) out[i] = 0.0;
    for (int i = 0; i <= 2 * ra; i++)
        for (int j = 0; j <= 2 * rb; j++) out[i + j] += a[i] * b[j];
}

void or_cdf97(double* h, double* g) {
    /* real root of 20y^3 + 10y^2 + 4y + 1 by Newton iteration */
    double y0 = -0.34;
    for (int it = 0; it < 100; it++) {
        double f = ((20.0 * y0 + 10.0) * y0 + 4.0) * y0 + 1.0;
        double df = (60.0 * y0 + 20.0) * y0 + 4.0;
        y0 -= f / df;
    }
    double q1 = 4.0 + 1.0 / y0, q2 = 10.0 + q1 / y0;
    double one_minus_y[3] = {0.25, 0.5, 0.25};
    double yv[3] = {-0.25, 0.5, -0.25};
    double sq[5], ysq[5], t5[5], t9[9], t7[7];
    lpoly_mul(one_minus_y, 1, one_minus_y, 1, sq);        /* (1-y)^2 */
    lpoly_mul(yv, 1, yv, 1, ysq);                          /* y^2     */
    /* q(y) = 1 + q1 y + q2 y^2 as taps -2..2 */
    for (int i = 0; i < 5; i++) t5[i] = q2 * ysq[i];
    for (int i = 0; i < 3; i++) t5[i + 1] += q1 * yv[i];
    t5[2] += 1.0;
    lpoly_mul(sq, 2, t5, 2, t9);
    /* r(y) = 1 - y/y0 */
    double r3[3];
    for (int i = 0; i < 3; i++) r3[i] = -yv[i] / y0;
    r3[1] += 1.0;
    lpoly_mul(sq, 2, r3, 1, t7);
    for (int i = 0; i < 9; i++) h[i] = sqrt(2.0) * t9[i];
    for (int i = 0; i < 7; i++) g[i] = sqrt(2.0) * t7[i];
}

static double g_h[9], g_g[7];
static int g_taps_ready = 0;
static void taps_init(void) {
    if (!g_taps_ready) { or_cdf97(g_h, g_g); g_taps_ready = 1; }
}

/* --------------------------------------------------- Laplacian pyramid
 * §2.1, Fig. 1: one LP level splits x into a lowpass c at half resolution
 * and a detail d at full resolution.  With periodic extension:
 *   down(x, f)[m][n] = sum_{a,b} f[a] f[b] x[2m-a][2n-b]          (filter, decimate)
 *   up(v, f)[y][x]   = sum_{m,n} f[y-2m] f[x-2n] v[m][n]          (expand, filter)
 * analysis:   c = down(x, h),  d = x - up(c, g)
 * synthesis:  x = d + up(c - down(d, h), g)        (dual-frame reading)
 * The separable sums are taken row pass first, then column pass.            */
static void down_filter(const double* x, int H, int W, const double* f, int R, double* out) {
    int Hh = H / 2, Wh = W / 2;
    double* t = (double*)malloc(sizeof(double) * (size_t)H * Wh);
    for (int r = 0; r < H; r++)
        for (int n = 0; n < Wh; n++) {
            double s = 0.0;
            for (int b = -R; b <= R; b++) s += f[b + R] * x[(long)r * W + wrapi(2L * n - b, W)];
            t[(long)r * Wh + n] = s;
        }
    for (int m = 0; m < Hh; m++)
        for (int n = 0; n < Wh; n++) {
            double s = 0.0;
            for (int a = -R; a <= R; a++) s += f[a + R] * t[(long)wrapi(2L * m - a, H) * Wh + n];
            out[(long)m * Wh + n] = s;
        }
    free(t);
}

static void up_filter(const double* v, int Hh, int Wh, const double* f, int R, double* out) {
    int H = 2 * Hh, W = 2 * Wh;
    double* t = (double*)malloc(sizeof(double) * (size_t)Hh * W);
    for (int m = 0; m < Hh; m++)
        for (int x = 0; x < W; x++) {
            double s = 0.0;
            for (int tt = -R; tt <= R; tt++) {
                int u = wrapi((long)x - tt, W);
                if ((u & 1) == 0) s += f[tt + R] * v[(long)m * Wh + u / 2];
            }
            t[(long)m * W + x] = s;
        }
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            double s = 0.0;
            for (int tt = -R; tt <= R; tt++) {
                int u = wrapi((long)y - tt, H);
                if ((u & 1) == 0) s += f[tt + R] * t[(long)(u / 2) * W + x];
            }
            out[(long)y * W + x] = s;
        }
    free(t);
}

void or_lp_analysis(const double* x, int H, int W, double* c, double* d) {
    taps_init();
    long n = (long)H * W;
    double* p = (double*)malloc(sizeof(double) * n);
    down_filter(x, H, W, g_h, 4, c);
    up_filter(c, H / 2, W / 2, g_g, 3, p);
    for (long i = 0; i < n; i++) d[i] = x[i] - p[i];
    free(p);
}

void or_lp_synthesis(const double* c, const double* d, int H, int W, double* x) {
    taps_init();
    long n = (long)H * W, nh = n / 4;
    double* e = (double*)malloc(sizeof(double) * nh);
    double* p = (double*)malloc(sizeof(double) * n);
    down_filter(d, H, W, g_h, 4, e);
    for (long i = 0; i < nh; i++) e[i] = c[i] - e[i];
    up_filter(e, H / 2, W / 2, g_g, 3, p);
    for (long i = 0; i < n; i++) x[i] = d[i] + p[i];
    free(e); free(p);
}

/* adjoint of the analysis map x -> (c, d):  xbar = dbar + up(cbar - down(dbar, g), h)
 * (down(., f) and up(., f) are each other's transposes for a symmetric f)    */
void or_lp_analysis_adjoint(const double* cbar, const double* dbar, int H, int W, double* xbar) {
    taps_init();
    long n = (long)H * W, nh = n / 4;
    double* e = (double*)malloc(sizeof(double) * nh);
    double* p = (double*)malloc(sizeof(double) * n);
    down_filter(dbar, H, W, g_g, 3, e);
    for (long i = 0; i < nh; i++) e[i] = cbar[i] - e[i];
    up_filter(e, H / 2, W / 2, g_h, 4, p);
    for (long i = 0; i < n; i++) xbar[i] = dbar[i] + p[i];
    free(e); free(p);
}

/* adjoint of the synthesis map (c, d) -> x:  cbar = down(xbar, g), dbar = xbar - up(cbar, h) */
void or_lp_synthesis_adjoint(const double* xbar, int H, int W, double* cbar, double* dbar) {
    taps_init();
    long n = (long)H * W;
    double* p = (double*)malloc(sizeof(double) * n);
    down_filter(xbar, H, W, g_g, 3, cbar);
    up_filter(cbar, H / 2, W / 2, g_h, 4, p);
    for (long i = 0; i < n; i++) dbar[i] = xbar[i] - p[i];
    free(p);
}

/* ------------------------------------------------ directional filter bank
 * §2.1: a DFB of l stages splits the detail image into 2^l wedge-shaped
 * subbands with perfect reconstruction.  Reading taken here:
 *
 * Stage building block: a two-channel fan filter bank on a channel's sample
 * lattice, written in lifting (ladder) form.  A channel is the coset
 * o + {b1*p1 + b2*p2} of the periodic H x W grid; in its coordinates p the
 * even samples (p1+p2 even) and the odd samples (p1+p2 odd) are the two
 * outputs.  With the 4-tap half-band prototype beta = (-1, 9, 9, -1)/16 at
 * a = -3,-1,1,3 modulated to the fan (betat[a] = (-1)^((a-1)/2) beta[a],
 * i.e. (-1, -9, 9, 1)/16) and the 16 neighbour offsets
 *   delta(a,b) = ((a+b)/2, (a-b)/2),  weight w = betat[a] * betat[b],
 *   predict (odd):  y = (x - sum_w x[p + delta]) / 2
 *   update (even):  y = x + sum_w y[p + delta]
 * (offsets in grid units: delta1*b1 + delta2*b2, wrapped periodically).
 *
 * Tree: stage 1 works in grid coordinates (b1=(1,0), b2=(0,1)); its even
 * output holds the fan |w_c| > |w_r| ("F_c"), its odd output (origin (1,0))
 * the fan |w_r| > |w_c| ("F_r").  From stage 2 on, a channel whose wedge
 * covers slopes [i/2^m, (i+1)/2^m] (F_c: slope w_r/w_c; F_r: slope w_c/w_r)
 * is split in the basis whose vectors are normal to the wedge's two edges,
 * so that the split line (the wedge bisector in slope) becomes the fan
 * diagonal:
 *   stage 2:  F_c  b1=(1,1),  b2=(1,-1);   F_r  b1=(1,1),  b2=(-1,1)
 *   stage s>=3, q = 2^(s-2):
 *             F_c  b1=(q,-2i), b2=(q,-2i-2);  F_r  b1=(-2i,q), b2=(-2i-2,q)
 * The even child takes the lower half of the slope range (index 2i), the odd
 * child (origin o + b1) the upper half (2i+1); after stage 2 the F_c / F_r
 * children carry i = -1, 0.  The final subbands are laid out on their
 * rectangular lattices: F_c on 2^(k-1) x 2 (rows x columns), F_r on
 * 2 x 2^(k-1); k = 1 keeps the two quincunx halves row-compacted.
 * Subband order = tree order (even child first at every split).            */
/* Longer prototypes (the PKVA structure admits any half-band beta): the
 * Lagrange (maximally flat) half-band interpolators of 6 and 8 taps,
 *   beta6 = (3, -25, 150, 150, -25, 3) / 256,
 *   beta8 = (-5, 49, -245, 1225, 1225, -245, 49, -5) / 2048,
 * at a = -5..5 and -7..7 (odd), modulated to the fan the same way.        */
static const int DFB_A[8] = {-7, -5, -3, -1, 1, 3, 5, 7};
static const double DFB_BETA4[4] = {-1.0 / 16, 9.0 / 16, 9.0 / 16, -1.0 / 16};
static const double DFB_BETA6[6] = {3.0 / 256, -25.0 / 256, 150.0 / 256, 150.0 / 256, -25.0 / 256, 3.0 / 256};
static const double DFB_BETA8[8] = {-5.0 / 2048, 49.0 / 2048, -245.0 / 2048, 1225.0 / 2048,
                                    1225.0 / 2048, -245.0 / 2048, 49.0 / 2048, -5.0 / 2048};

/* the fan taps betat[a] = (-1)^((a-1)/2) beta[a] of an n-tap prototype, at
 * offsets a = DFB_A[4 - n/2 ..]; 0 unless n is 4, 6 or 8 */
static int dfb_taps(int n, const int** a, double* bt) {
    const double* beta = n == 4 ? DFB_BETA4 : (n == 6 ? DFB_BETA6 : (n == 8 ? DFB_BETA8 : NULL));
    if (!beta) return 0;
    *a = DFB_A + 4 - n / 2;
    for (int t = 0; t < n; t++) {
        int av = (*a)[t];
        int e = (av - 1) / 2;                         /* exact: av is odd */
        bt[t] = ((e % 2 + 2) % 2 ? -1.0 : 1.0) * beta[t];
    }
    return n;
}

typedef struct { int o_r, o_c, T, i; } dfb_chan; /* T: 0 = F_c, 1 = F_r */

static void dfb_basis(int s, const dfb_chan* ch, int* b /* b1r b1c b2r b2c */) {
    if (s == 1) { b[0] = 1; b[1] = 0; b[2] = 0; b[3] = 1; return; }
    if (s == 2) {
        if (ch->T == 0) { b[0] = 1; b[1] = 1; b[2] = 1; b[3] = -1; }
        else { b[0] = 1; b[1] = 1; b[2] = -1; b[3] = 1; }
        return;
    }
    int q = 1 << (s - 2), i = ch->i;
    if (ch->T == 0) { b[0] = q; b[1] = -2 * i; b[2] = q; b[3] = -2 * i - 2; }
    else { b[0] = -2 * i; b[1] = q; b[2] = -2 * i - 2; b[3] = q; }
}

static void dfb_children(int s, const dfb_chan* ch, const int* b, dfb_chan* c0, dfb_chan* c1) {
    c0->o_r = ch->o_r; c0->o_c = ch->o_c;
    c1->o_r = ch->o_r + b[0]; c1->o_c = ch->o_c + b[1];
    if (s == 1) { c0->T = 0; c1->T = 1; c0->i = c1->i = 0; }
    else if (s == 2) { c0->T = c1->T = ch->T; c0->i = -1; c1->i = 0; }
    else { c0->T = c1->T = ch->T; c0->i = 2 * ch->i; c1->i = 2 * ch->i + 1; }
}

typedef struct {
    int H, W, k;
    dfb_chan* chans[OR_MAX_K + 2];  /* chans[s]: 2^(s-1) input channels of stage s; chans[k+1]: final */
    unsigned char* par[OR_MAX_K + 1]; /* par[s][pixel]: parity in its stage-s channel */
    int* cid[OR_MAX_K + 1];           /* cid[s][pixel]: stage-s channel index          */
} dfb_plan;

static void dfb_plan_make(dfb_plan* P, int H, int W, int k) {
    memset(P, 0, sizeof(*P));
    P->H = H; P->W = W; P->k = k;
    P->chans[1] = (dfb_chan*)calloc(1, sizeof(dfb_chan));
    for (int s = 1; s <= k; s++) {
        int n = 1 << (s - 1);
        P->chans[s + 1] = (dfb_chan*)calloc((size_t)2 * n, sizeof(dfb_chan));
        for (int c = 0; c < n; c++) {
            int b[4];
            dfb_basis(s, &P->chans[s][c], b);
            dfb_children(s, &P->chans[s][c], b, &P->chans[s + 1][2 * c], &P->chans[s + 1][2 * c + 1]);
        }
    }
    long np = (long)H * W;
    for (int s = 1; s <= k; s++) {
        P->par[s] = (unsigned char*)malloc((size_t)np);
        P->cid[s] = (int*)malloc(sizeof(int) * (size_t)np);
    }
    for (int r = 0; r < H; r++)
        for (int c = 0; c < W; c++) {
            long idx = (long)r * W + c;
            int ch = 0;
            for (int s = 1; s <= k; s++) {
                const dfb_chan* C = &P->chans[s][ch];
                int b[4];
                dfb_basis(s, C, b);
                long det = (long)b[0] * b[3] - (long)b[1] * b[2];
                long dr = r - C->o_r, dc = c - C->o_c;
                long n1 = (long)b[3] * dr - (long)b[2] * dc;
                long n2 = -(long)b[1] * dr + (long)b[0] * dc;
                /* the pixel lies on this channel's lattice: both divisions are exact */
                if (n1 % det != 0 || n2 % det != 0) abort();
                long p1 = n1 / det, p2 = n2 / det;
                int parity = (int)(((p1 + p2) % 2 + 2) % 2);
                P->par[s][idx] = (unsigned char)parity;
                P->cid[s][idx] = ch;
                ch = 2 * ch + parity;
            }
        }
}

static void dfb_plan_free(dfb_plan* P) {
    for (int s = 1; s <= P->k + 1; s++) free(P->chans[s]);
    for (int s = 1; s <= P->k; s++) { free(P->par[s]); free(P->cid[s]); }
}

/* one lifting pass of stage s: every sample of parity `target` becomes
 * alpha * itself + gamma * (weighted sum of its n^2 neighbours of the other parity) */
static void dfb_pass(const dfb_plan* P, double* x, int s, int target, double alpha, double gamma, int n,
                     const int* A, const double* BT) {
    int H = P->H, W = P->W;
    for (int r = 0; r < H; r++)
        for (int c = 0; c < W; c++) {
            long idx = (long)r * W + c;
            if (P->par[s][idx] != target) continue;
            int b[4];
            dfb_basis(s, &P->chans[s][P->cid[s][idx]], b);
            double acc = 0.0;
            for (int ia = 0; ia < n; ia++)
                for (int ib = 0; ib < n; ib++) {
                    int a = A[ia], bb = A[ib];
                    int d1 = (a + bb) / 2, d2 = (a - bb) / 2;
                    int orr = d1 * b[0] + d2 * b[2], occ = d1 * b[1] + d2 * b[3];
                    acc += BT[ia] * BT[ib] * x[(long)wrapi((long)r + orr, H) * W + wrapi((long)c + occ, W)];
                }
            x[idx] = alpha * x[idx] + gamma * acc;
        }
}

/* position of element (a, b) of final subband `ci` in the detail image */
static void dfb_leaf_pos(const dfb_plan* P, int ci, int a, int b, int* r, int* c) {
    int k = P->k, H = P->H, W = P->W;
    if (k == 0) { *r = a; *c = b; return; }
    const dfb_chan* C = &P->chans[k + 1][ci];
    if (k == 1) { *r = a; *c = 2 * b + ((a + C->o_r + C->o_c) & 1); return; }
    int R = C->T == 0 ? (1 << (k - 1)) : 2;
    int Cc = C->T == 0 ? 2 : (1 << (k - 1));
    *r = wrapi((long)wrapi(C->o_r, R) + (long)R * a, H);
    *c = wrapi((long)wrapi(C->o_c, Cc) + (long)Cc * b, W);
}

static void dfb_leaf_dims(const dfb_plan* P, int ci, int* h, int* w) {
    int k = P->k, H = P->H, W = P->W;
    if (k == 0) { *h = H; *w = W; return; }
    if (k == 1) { *h = H; *w = W / 2; return; }
    if (P->chans[k + 1][ci].T == 0) { *h = H >> (k - 1); *w = W / 2; }
    else { *h = H / 2; *w = W >> (k - 1); }
}

int or_dfb(int mode, const double* in, int H, int W, int k, double* out) {
    return or_dfb_taps(mode, in, H, W, k, 4, out);
}

int or_dfb_taps(int mode, const double* in, int H, int W, int k, int taps, double* out) {
    const int* A;
    double BT[8];
    int n = dfb_taps(taps, &A, BT);
    if (!n || k < 0 || k > OR_MAX_K) return OR_EINVAL;
    int need = k >= 2 ? (1 << (k - 1)) : 2;
    if (k > 0 && (H % need || W % need)) return OR_EINVAL;
    long np = (long)H * W;
    if (k == 0) { memcpy(out, in, sizeof(double) * np); return OR_OK; }
    dfb_plan P;
    dfb_plan_make(&P, H, W, k);
    double* x = (double*)malloc(sizeof(double) * np);
    int nl = 1 << k;
    if (mode == 0 || mode == 3) {
        /* analysis direction, stages 1..k */
        memcpy(x, in, sizeof(double) * np);
        for (int s = 1; s <= k; s++) {
            if (mode == 0) {            /* forward: predict odd, then update even */
                dfb_pass(&P, x, s, 1, 0.5, -0.5, n, A, BT);
                dfb_pass(&P, x, s, 0, 1.0, 1.0, n, A, BT);
            } else {                    /* transpose of the inverse stage */
                dfb_pass(&P, x, s, 0, 1.0, 1.0, n, A, BT);
                dfb_pass(&P, x, s, 1, 2.0, -1.0, n, A, BT);
            }
        }
        long o = 0;
        for (int ci = 0; ci < nl; ci++) {
            int h, w;
            dfb_leaf_dims(&P, ci, &h, &w);
            for (int a = 0; a < h; a++)
                for (int b = 0; b < w; b++) {
                    int r, c;
                    dfb_leaf_pos(&P, ci, a, b, &r, &c);
                    out[o++] = x[(long)r * W + c];
                }
        }
    } else {
        /* synthesis direction, stages k..1 */
        long o = 0;
        for (int ci = 0; ci < nl; ci++) {
            int h, w;
            dfb_leaf_dims(&P, ci, &h, &w);
            for (int a = 0; a < h; a++)
                for (int b = 0; b < w; b++) {
                    int r, c;
                    dfb_leaf_pos(&P, ci, a, b, &r, &c);
                    x[(long)r * W + c] = in[o++];
                }
        }
        for (int s = k; s >= 1; s--) {
            if (mode == 1) {            /* inverse: undo update, then undo predict */
                dfb_pass(&P, x, s, 0, 1.0, -1.0, n, A, BT);
                dfb_pass(&P, x, s, 1, 2.0, 1.0, n, A, BT);
            } else {                    /* transpose of the forward stage */
                dfb_pass(&P, x, s, 1, 0.5, 0.5, n, A, BT);
                dfb_pass(&P, x, s, 0, 1.0, -1.0, n, A, BT);
            }
        }
        memcpy(out, x, sizeof(double) * np);
    }
    free(x);
    dfb_plan_free(&P);
    return OR_OK;
}

/* ------------------------------------------------- contourlet transform
 * §2.1 / Fig. 1: the LP is iterated on the lowpass; every LP detail d_j
 * feeds a DFB with k_j stages.  Modes: 0 forward A, 1 inverse S,
 * 2 adjoint A^T, 3 adjoint S^T.                                             */
int or_ct(int mode, const double* in, int H, int W, int L, const int* k, double* out) {
    return or_ct_taps(mode, in, H, W, L, k, 4, out);
}

int or_ct_taps(int mode, const double* in, int H, int W, int L, const int* k, int taps, double* out) {
    or_layout lay;
    int st = or_layout_make(H, W, L, k, &lay);
    if (st) return st;
    double* cur = (double*)malloc(sizeof(double) * (size_t)H * W);
    double* det = (double*)malloc(sizeof(double) * (size_t)H * W);
    double* nxt = (double*)malloc(sizeof(double) * (size_t)H * W);
    if (mode == 0 || mode == 3) {
        memcpy(cur, in, sizeof(double) * (size_t)H * W);
        long off = lay.sb[0].h * (long)lay.sb[0].w;
        for (int j = 1; j <= L; j++) {
            int Hj = H >> (j - 1), Wj = W >> (j - 1);
            if (mode == 0) or_lp_analysis(cur, Hj, Wj, nxt, det);
            else or_lp_synthesis_adjoint(cur, Hj, Wj, nxt, det);
            st = or_dfb_taps(mode, det, Hj, Wj, k[j - 1], taps, out + off);
            if (st) break;
            off += (long)Hj * Wj;
            double* t = cur; cur = nxt; nxt = t;
        }
        memcpy(out, cur, sizeof(double) * lay.sb[0].h * (long)lay.sb[0].w);
    } else {
        memcpy(cur, in, sizeof(double) * lay.sb[0].h * (long)lay.sb[0].w);
        long offs[OR_MAX_LEVELS + 1];
        long off = lay.sb[0].h * (long)lay.sb[0].w;
        for (int j = 1; j <= L; j++) { offs[j] = off; off += (long)(H >> (j - 1)) * (W >> (j - 1)); }
        for (int j = L; j >= 1; j--) {
            int Hj = H >> (j - 1), Wj = W >> (j - 1);
            st = or_dfb_taps(mode, in + offs[j], Hj, Wj, k[j - 1], taps, det);
            if (st) break;
            if (mode == 1) or_lp_synthesis(cur, det, Hj, Wj, nxt);
            else or_lp_analysis_adjoint(cur, det, Hj, Wj, nxt);
            double* t = cur; cur = nxt; nxt = t;
        }
        memcpy(out, cur, sizeof(double) * (size_t)H * W);
    }
    free(cur); free(det); free(nxt);
    return st;
}

/* --------------------------------------------------------------- colour
 * Table 1 (Eq. 1-6) in its integer lifting form YCoCg-R (lossless):
 *   Co = R - B,  t = B + floor(Co/2),  Cg = G - t,  Y = t + floor(Cg/2)
 *   t = Y - floor(Cg/2),  G = Cg + t,  B = t - floor(Co/2),  R = B + Co
 * Decoded values are clamped to [0, 255].                                   */
void or_ycocgr_forward(const uint8_t* rgb, long n, int16_t* y, int16_t* co, int16_t* cg) {
    for (long i = 0; i < n; i++) {
        long R = rgb[3 * i], G = rgb[3 * i + 1], B = rgb[3 * i + 2];
        long Co = R - B;
        long t = B + floordiv(Co, 2);
        long Cg = G - t;
        long Y = t + floordiv(Cg, 2);
        y[i] = (int16_t)Y; co[i] = (int16_t)Co; cg[i] = (int16_t)Cg;
    }
}

static int clampi(long v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : (int)v); }

void or_ycocgr_inverse(const int16_t* y, const int16_t* co, const int16_t* cg, long n, uint8_t* rgb) {
    for (long i = 0; i < n; i++) {
        long t = (long)y[i] - floordiv(cg[i], 2);
        long G = cg[i] + t;
        long B = t - floordiv(co[i], 2);
        long R = B + co[i];
        rgb[3 * i] = (uint8_t)clampi(R, 0, 255);
        rgb[3 * i + 1] = (uint8_t)clampi(G, 0, 255);
        rgb[3 * i + 2] = (uint8_t)clampi(B, 0, 255);
    }
}

/* v / d for d = 2 or 4, rounded half away from zero (exact integer arithmetic) */
static long div_round(long v, long d) {
    long a = v < 0 ? -v : v;
    a = (a + d / 2) / d;
    return v < 0 ? -a : a;
}

void or_ycocg8_forward(const uint8_t* rgb, long n, int16_t* y, int16_t* co, int16_t* cg) {
    for (long i = 0; i < n; i++) {
        long R = rgb[3 * i], G = rgb[3 * i + 1], B = rgb[3 * i + 2];
        y[i] = (int16_t)div_round(R + 2 * G + B, 4);
        co[i] = (int16_t)clampi(div_round(R - B, 2) + 127, 0, 255);
        cg[i] = (int16_t)clampi(div_round(2 * G - R - B, 4) + 127, 0, 255);
    }
}

void or_ycocg8_inverse(const int16_t* y, const int16_t* co, const int16_t* cg, long n, uint8_t* rgb) {
    for (long i = 0; i < n; i++) {
        long Y = y[i], Co = (long)co[i] - 127, Cg = (long)cg[i] - 127;
        rgb[3 * i] = (uint8_t)clampi(Y + Co - Cg, 0, 255);
        rgb[3 * i + 1] = (uint8_t)clampi(Y + Cg, 0, 255);
        rgb[3 * i + 2] = (uint8_t)clampi(Y - Co - Cg, 0, 255);
    }
}

/* §3.1 chroma subsampling, factor N = 4 read as 2 x 2: rounded mean of each
 * 2x2 block, floor((s + 2) / 4); odd sizes replicate the last row / column. */
void or_chroma_down(const int16_t* in, int H, int W, int16_t* out) {
    int Hc = (H + 1) / 2, Wc = (W + 1) / 2;
    for (int i = 0; i < Hc; i++)
        for (int j = 0; j < Wc; j++) {
            int r0 = 2 * i, r1 = 2 * i + 1 < H ? 2 * i + 1 : H - 1;
            int c0 = 2 * j, c1 = 2 * j + 1 < W ? 2 * j + 1 : W - 1;
            long s = (long)in[(long)r0 * W + c0] + in[(long)r0 * W + c1] + in[(long)r1 * W + c0] + in[(long)r1 * W + c1];
            out[(long)i * Wc + j] = (int16_t)floordiv(s + 2, 4);
        }
}

/* §3.1 decoder: bilinear interpolation from the four neighbouring chroma
 * samples.  Centred siting: full-resolution row y sits at chroma row
 * (y - 1/2)/2, so even rows weigh rows (i-1, i) by (1/4, 3/4) and odd rows
 * rows (i, i+1) by (3/4, 1/4); indices clamp at the edges.  2-D weights
 * (9,3,3,1)/16 with rounding: floor((9a + 3b + 3c + d + 8) / 16).           */
void or_chroma_up(const int16_t* in, int Hc, int Wc, int H, int W, int16_t* out) {
    for (int y = 0; y < H; y++) {
        int i0 = y / 2, i1 = (y & 1) ? i0 + 1 : i0 - 1;
        if (i1 < 0) i1 = 0;
        if (i1 > Hc - 1) i1 = Hc - 1;
        if (i0 > Hc - 1) i0 = Hc - 1;
        for (int x = 0; x < W; x++) {
            int j0 = x / 2, j1 = (x & 1) ? j0 + 1 : j0 - 1;
            if (j1 < 0) j1 = 0;
            if (j1 > Wc - 1) j1 = Wc - 1;
            if (j0 > Wc - 1) j0 = Wc - 1;
            long s = 9L * in[(long)i0 * Wc + j0] + 3L * in[(long)i1 * Wc + j0] + 3L * in[(long)i0 * Wc + j1] + in[(long)i1 * Wc + j1];
            out[(long)y * W + x] = (int16_t)floordiv(s + 8, 16);
        }
    }
}

/* plane padding to the layout modulus: half-sample symmetric mirror at the
 * bottom and right edges, x[H + i] = x[H - 1 - i] (the paper is silent).   */
void or_pad_mirror(const double* in, int H, int W, int Hp, int Wp, double* out) {
    for (int r = 0; r < Hp; r++) {
        int sr = r < H ? r : 2 * H - 1 - r;
        for (int c = 0; c < Wp; c++) {
            int sc = c < W ? c : 2 * W - 1 - c;
            out[(long)r * Wp + c] = in[(long)sr * W + sc];
        }
    }
}

/* ------------------------------------------------------------ quantiser
 * §3.5 divide by QPH (subbands) or QPL (lowpass), §3.6 round to the nearest
 * integer (ties away from zero).  The lowpass is first normalised (§3.4) by
 * the exact factor 2^-L; subband coefficients below the threshold magnitude
 * are set to zero first.  Decision in single precision; |q| > 32767 is an
 * overflow of the int16 code.                                               */
int or_quantize(float c, int qp, float threshold, int is_lowpass, int levels, int* ovf) {
    float t;
    if (is_lowpass) t = ldexpf(c, -levels);
    else t = (fabsf(c) >= threshold) ? c : 0.0f;
    float v = roundf(t / (float)qp);
    if (!(fabsf(v) <= 32767.0f)) { *ovf = 1; return 0; }
    return (int)v;
}

int or_quantize8(float c, int qp, float threshold, int is_lowpass, int levels) {
    float t;
    if (is_lowpass) t = ldexpf(c, -levels);
    else t = (fabsf(c) >= threshold) ? c : 0.0f;
    float v = roundf(t / (float)qp);                 /* §3.5 divide, §3.6 round: one rounding */
    float lo = is_lowpass ? 0.0f : -128.0f, hi = is_lowpass ? 255.0f : 127.0f;
    if (v < lo) v = lo;                              /* §3.6: the code is kept in a byte */
    if (v > hi) v = hi;
    return (int)v;
}

/* ---------------------------------------------------- soft thresholding */
static double or_sign(double v) { return v > 0.0 ? 1.0 : (v < 0.0 ? -1.0 : 0.0); }

void or_soft_threshold(const double* c, const or_layout* lay, int batch, const double* T, double* y) {
    for (int b = 0; b < batch; b++) {
        const double* cb = c + (long)b * lay->total;
        double* yb = y + (long)b * lay->total;
        for (int s = 0; s < lay->nsub; s++) {
            const or_subband* sb = &lay->sb[s];
            for (long e = 0; e < (long)sb->h * sb->w; e++) {
                double v = cb[sb->off + e];
                if (s == 0) yb[sb->off + e] = v;
                else yb[sb->off + e] = or_sign(v) * fmax(fabs(v) - T[s - 1], 0.0);
            }
        }
    }
}

void or_soft_threshold_vjp(const double* c, const or_layout* lay, int batch, const double* T, const double* g,
                           double* gc, double* gT) {
    for (int s = 0; s + 1 < lay->nsub; s++) gT[s] = 0.0;
    for (int b = 0; b < batch; b++) {
        long base = (long)b * lay->total;
        for (int s = 0; s < lay->nsub; s++) {
            const or_subband* sb = &lay->sb[s];
            for (long e = 0; e < (long)sb->h * sb->w; e++) {
                long i = base + sb->off + e;
                if (s == 0) { gc[i] = g[i]; continue; }
                int on = fabs(c[i]) > T[s - 1];
                gc[i] = on ? g[i] : 0.0;
                if (on) gT[s - 1] -= g[i] * or_sign(c[i]);
            }
        }
    }
}

/* ------------------------------------------------------------------ RLE
 * §3.8: zero runs are coded along the horizontal direction; rows are coded
 * independently.  A non-zero value v is the token v; a maximal run of n
 * zeros is the token pair (0, n).                                           */
long or_rle_row(const int16_t* row, int w, int16_t* tokens) {
    long n = 0;
    int x = 0;
    while (x < w) {
        if (row[x] != 0) { tokens[n++] = row[x]; x++; continue; }
        int run = 0;
        while (x < w && row[x] == 0) { run++; x++; }
        tokens[n++] = 0;
        tokens[n++] = (int16_t)run;
    }
    return n;
}

int or_rle_expand(const int16_t* tokens, long ntok, int16_t* out, long n) {
    long pos = 0, t = 0;
    while (t < ntok) {
        if (tokens[t] != 0) {
            if (pos >= n) return OR_ECORRUPT;
            out[pos++] = tokens[t++];
            continue;
        }
        if (t + 1 >= ntok) return OR_ECORRUPT;
        long run = tokens[t + 1];
        if (run <= 0 || pos + run > n) return OR_ECORRUPT;
        for (long i = 0; i < run; i++) out[pos++] = 0;
        t += 2;
    }
    return pos == n ? OR_OK : OR_ECORRUPT;
}

/* ---------------------------------------------------------------- codec */
struct or_codec {
    int Wo, Ho, L, k[OR_MAX_LEVELS], qph, qpl, kint;
    float thr;
    int Hp, Wp, Hc, Wc, Hcp, Wcp;
    or_layout ly, lc;
    long ncoef;
    int ncomp;
    int16_t* enc_state;
    int16_t* dec_state;
    long enc_frame;
    long dec_next;  /* index the next P-frame must carry; -1: a K-frame is required */
    int dec_floor;  /* finest levels 1..dec_floor of the decoder state are missing */
    int range;      /* motion search range W (0: zero-motion P-frames) */
    int nby, nbx;   /* 16 x 16 luma blocks */
    uint8_t* enc_luma;   /* the previous frame's padded luma (encoder) */
    int st8;        /* 8-bit storage (§3.1, §3.6) */
    int taps;       /* DFB prototype length: 4, 6 or 8 */
};

static int round_up(int v, int m) { return (v + m - 1) / m * m; }

or_codec* or_codec_create(int width, int height, int levels, const int* dirs, int qph, int qpl,
                          float threshold, int key_interval) {
    if (width <= 0 || height <= 0 || width > 65535 || height > 65535) return NULL;
    if (levels < 1 || levels > OR_MAX_LEVELS) return NULL;
    if (qph < 1 || qph > 181 || qpl < 1 || qpl > 71 || key_interval < 1) return NULL;
    if (!(threshold >= 0.0f)) return NULL;
    or_codec* c = (or_codec*)calloc(1, sizeof(or_codec));
    c->Wo = width; c->Ho = height; c->L = levels; c->qph = qph; c->qpl = qpl;
    c->thr = threshold; c->kint = key_interval; c->taps = 4;
    for (int j = 0; j < levels; j++) c->k[j] = dirs[j];
    int M = or_modulus(levels, c->k);
    c->Hp = round_up(height, M); c->Wp = round_up(width, M);
    c->Hc = (height + 1) / 2; c->Wc = (width + 1) / 2;
    c->Hcp = round_up(c->Hc, M); c->Wcp = round_up(c->Wc, M);
    /* the mirror reaches back at most one plane height */
    if (c->Hp > 2 * height || c->Wp > 2 * width || c->Hcp > 2 * c->Hc || c->Wcp > 2 * c->Wc ||
        or_layout_make(c->Hp, c->Wp, levels, c->k, &c->ly) ||
        or_layout_make(c->Hcp, c->Wcp, levels, c->k, &c->lc)) {
        free(c);
        return NULL;
    }
    c->ncoef = c->ly.total + 2 * c->lc.total;
    c->ncomp = c->ly.nsub + 2 * c->lc.nsub;
    c->enc_state = (int16_t*)calloc((size_t)c->ncoef, sizeof(int16_t));
    c->dec_state = (int16_t*)calloc((size_t)c->ncoef, sizeof(int16_t));
    or_codec_reset(c);
    return c;
}

void or_codec_destroy(or_codec* c) {
    if (!c) return;
    free(c->enc_state); free(c->dec_state); free(c->enc_luma); free(c);
}

int or_codec_set_motion(or_codec* c, int range) {
    if (range < 0 || range > OR_MAX_RANGE) return OR_EINVAL;
    c->range = range;
    c->nby = (c->Hp + 15) / 16;
    c->nbx = (c->Wp + 15) / 16;
    free(c->enc_luma);
    c->enc_luma = range ? (uint8_t*)calloc((size_t)c->Hp * c->Wp, 1) : NULL;
    return OR_OK;
}

int or_codec_set_storage8(or_codec* c, int on) {
    c->st8 = on != 0;
    return OR_OK;
}

int or_codec_set_taps(or_codec* c, int taps) {
    if (taps != 4 && taps != 6 && taps != 8) return OR_EINVAL;
    c->taps = taps;
    return OR_OK;
}

/* header byte 5: bit 0 the 8-bit storage, bits 1-2 the DFB prototype (0: 4 taps, 1: 6, 2: 8) */
static int flags_byte(const or_codec* c) { return c->st8 | ((c->taps / 2 - 2) << 1); }

/* §3.2: full-search block matching on luma (see oracle.h) */
void or_motion_search(const uint8_t* cur, const uint8_t* prev, int H, int W, int range, int8_t* mv) {
    int nby = (H + 15) / 16, nbx = (W + 15) / 16;
    for (int by = 0; by < nby; by++)
        for (int bx = 0; bx < nbx; bx++) {
            int y0 = 16 * by, x0 = 16 * bx;
            int bh = H - y0 < 16 ? H - y0 : 16, bw = W - x0 < 16 ? W - x0 : 16;
            long best = -1;
            int bdy = 0, bdx = 0;
            for (int dy = -range; dy <= range; dy++)
                for (int dx = -range; dx <= range; dx++) {
                    if (y0 + dy < 0 || y0 + dy + bh > H || x0 + dx < 0 || x0 + dx + bw > W) continue;
                    long sse = 0;
                    for (int y = 0; y < bh; y++)
                        for (int x = 0; x < bw; x++) {
                            long d = (long)cur[(long)(y0 + y) * W + x0 + x] -
                                     (long)prev[(long)(y0 + dy + y) * W + x0 + dx + x];
                            sse += d * d;
                        }
                    int better = best < 0 || sse < best;
                    if (!better && sse == best) {
                        int m = abs(dy) + abs(dx), bm = abs(bdy) + abs(bdx);
                        better = m < bm;   /* equal norms: the earlier candidate stays */
                    }
                    if (better) { best = sse; bdy = dy; bdx = dx; }
                }
            mv[2 * (by * nbx + bx)] = (int8_t)bdy;
            mv[2 * (by * nbx + bx) + 1] = (int8_t)bdx;
        }
}
void or_codec_reset(or_codec* c) { c->enc_frame = 0; c->dec_next = -1; c->dec_floor = 0; }
long or_codec_coeff_count(const or_codec* c) { return c->ncoef; }
int or_codec_ncomp(const or_codec* c) { return c->ncomp; }
long or_codec_max_stream(const or_codec* c) {
    return 32 + 4L * c->ncomp + 2L * 2L * c->ncoef + (c->range ? 2L * c->nby * c->nbx : 0);
}
void or_codec_dims(const or_codec* c, int* out) { out[0] = c->Hp; out[1] = c->Wp; out[2] = c->Hcp; out[3] = c->Wcp; }

void or_codec_planes(const or_codec* c, const uint8_t* rgb, double* y, double* co, double* cg) {
    long n = (long)c->Ho * c->Wo, nc = (long)c->Hc * c->Wc;
    int16_t* Y = (int16_t*)malloc(sizeof(int16_t) * n);
    int16_t* Co = (int16_t*)malloc(sizeof(int16_t) * n);
    int16_t* Cg = (int16_t*)malloc(sizeof(int16_t) * n);
    int16_t* Co2 = (int16_t*)malloc(sizeof(int16_t) * nc);
    int16_t* Cg2 = (int16_t*)malloc(sizeof(int16_t) * nc);
    double* t = (double*)malloc(sizeof(double) * n);
    if (c->st8) or_ycocg8_forward(rgb, n, Y, Co, Cg);
    else or_ycocgr_forward(rgb, n, Y, Co, Cg);
    or_chroma_down(Co, c->Ho, c->Wo, Co2);
    or_chroma_down(Cg, c->Ho, c->Wo, Cg2);
    for (long i = 0; i < n; i++) t[i] = Y[i];
    or_pad_mirror(t, c->Ho, c->Wo, c->Hp, c->Wp, y);
    for (long i = 0; i < nc; i++) t[i] = Co2[i];
    or_pad_mirror(t, c->Hc, c->Wc, c->Hcp, c->Wcp, co);
    for (long i = 0; i < nc; i++) t[i] = Cg2[i];
    or_pad_mirror(t, c->Hc, c->Wc, c->Hcp, c->Wcp, cg);
    free(Y); free(Co); free(Cg); free(Co2); free(Cg2); free(t);
}

static void put16(uint8_t* p, unsigned v) { p[0] = (uint8_t)(v & 255); p[1] = (uint8_t)((v >> 8) & 255); }
static void put32(uint8_t* p, unsigned long v) { for (int i = 0; i < 4; i++) p[i] = (uint8_t)((v >> (8 * i)) & 255); }
static unsigned get16(const uint8_t* p) { return (unsigned)p[0] | ((unsigned)p[1] << 8); }
static unsigned long get32(const uint8_t* p) {
    return (unsigned long)p[0] | ((unsigned long)p[1] << 8) | ((unsigned long)p[2] << 16) | ((unsigned long)p[3] << 24);
}

/* component j of the frame: plane index and subband */
static const or_subband* comp_sb(const or_codec* c, int j, long* base) {
    if (j < c->ly.nsub) { *base = 0; return &c->ly.sb[j]; }
    j -= c->ly.nsub;
    int p = j / c->lc.nsub;
    *base = c->ly.total + p * c->lc.total;
    return &c->lc.sb[j % c->lc.nsub];
}

static int ilog2(long v) { int e = 0; while ((1L << e) < v) e++; return e; }

/* §3.7: the motion-compensated prediction of component j from the previous
 * frame's codes `prev` (whole-frame array).  One element of the component
 * stands for 2^ey x 2^ex luma samples (its plane's size over its own, times 2
 * for chroma); element (i, j) takes the vector of the luma block holding its
 * first luma sample (i 2^ey, j 2^ex), scaled to the component by 2^-ey, 2^-ex
 * and rounded half away from zero, and reads prev at the displaced element,
 * clamped to the component. */
static long rshift_round(long v, int e) {
    if (e == 0) return v;
    long a = v < 0 ? -v : v;
    a = (a + (1L << (e - 1))) >> e;
    return v < 0 ? -a : a;
}
static void mc_predict(const or_codec* c, int j, const int16_t* prev, const int8_t* mv, int16_t* pred) {
    long base;
    const or_subband* s = comp_sb(c, j, &base);
    int chroma = j >= c->ly.nsub;
    int ey = ilog2((chroma ? c->Hcp : c->Hp) / s->h) + chroma;
    int ex = ilog2((chroma ? c->Wcp : c->Wp) / s->w) + chroma;
    const int16_t* P = prev + base + s->off;
    int16_t* Q = pred + base + s->off;
    for (int i = 0; i < s->h; i++)
        for (int k = 0; k < s->w; k++) {
            long by = ((long)i << ey) >> 4, bx = ((long)k << ex) >> 4;
            if (by > c->nby - 1) by = c->nby - 1;
            if (bx > c->nbx - 1) bx = c->nbx - 1;
            const int8_t* v = mv + 2 * (by * c->nbx + bx);
            long si = i + rshift_round(v[0], ey), sk = k + rshift_round(v[1], ex);
            si = si < 0 ? 0 : (si > s->h - 1 ? s->h - 1 : si);
            sk = sk < 0 ? 0 : (sk > s->w - 1 ? s->w - 1 : sk);
            Q[(long)i * s->w + k] = P[si * s->w + sk];
        }
}

/* §3.7: frame i (counted from the last reset) is a K-frame iff i is a
 * multiple of the key interval.  K-frame: every lowpass column is replaced by
 * its first difference (each element minus the element above), subbands pass
 * unchanged.  P-frame: every component is the difference between the current
 * and the previous frame's codes (zero motion).  Differences wrap in 16 bits;
 * the coder state is the current frame's codes.  §3.8: K-frame lowpass is
 * stored raw, every other component is run-length coded.                    */
int or_encode_from_coeffs(or_codec* c, const float* coeffs, uint8_t* out, long cap,
                          long* out_len, int* frame_type) {
    if (c->range) return OR_EINVAL;   /* motion search needs the frame's luma */
    return or_encode_from_coeffs_luma(c, coeffs, NULL, out, cap, out_len, frame_type);
}

int or_encode_from_coeffs_luma(or_codec* c, const float* coeffs, const uint8_t* luma, uint8_t* out, long cap,
                               long* out_len, int* frame_type) {
    if (c->range && !luma) return OR_EINVAL;
    int type = (c->enc_frame % c->kint) == 0 ? 0 : (c->range ? 2 : 1);
    int16_t* q = (int16_t*)malloc(sizeof(int16_t) * (size_t)c->ncoef);
    int16_t* r = (int16_t*)malloc(sizeof(int16_t) * (size_t)c->ncoef);
    int ovf = 0;
    for (int j = 0; j < c->ncomp; j++) {
        long base;
        const or_subband* s = comp_sb(c, j, &base);
        int low = s->kind == 0;
        for (long e = 0; e < (long)s->h * s->w; e++) {
            long idx = base + s->off + e;
            int qp = low ? c->qpl : c->qph;
            q[idx] = (int16_t)(c->st8 ? or_quantize8(coeffs[idx], qp, c->thr, low, c->L)
                                      : or_quantize(coeffs[idx], qp, c->thr, low, c->L, &ovf));
        }
    }
    if (ovf) { free(q); free(r); return OR_EOVERFLOW; }
    /* P-frame with motion: the prediction of every component (§3.2, §3.7) */
    long nmv = (long)c->nby * c->nbx;
    int8_t* mv = NULL;
    int16_t* pred = NULL;
    if (type == 2) {
        mv = (int8_t*)malloc((size_t)(2 * nmv));
        pred = (int16_t*)malloc(sizeof(int16_t) * (size_t)c->ncoef);
        or_motion_search(luma, c->enc_luma, c->Hp, c->Wp, c->range, mv);
        for (int j = 0; j < c->ncomp; j++) mc_predict(c, j, c->enc_state, mv, pred);
    }
    for (int j = 0; j < c->ncomp; j++) {
        long base;
        const or_subband* s = comp_sb(c, j, &base);
        for (int a = 0; a < s->h; a++)
            for (int b = 0; b < s->w; b++) {
                long idx = base + s->off + (long)a * s->w + b;
                int v;
                if (type == 2) v = q[idx] - pred[idx];
                else if (type == 1) v = q[idx] - c->enc_state[idx];
                else if (s->kind == 0 && a > 0) v = q[idx] - q[idx - s->w];
                else v = q[idx];
                r[idx] = (int16_t)(uint16_t)(v & 0xFFFF);
            }
    }
    /* bitstream: 32-byte header, ncomp u32 token counts, int16 tokens */
    long need = 32 + 4L * c->ncomp;
    int16_t* tok = (int16_t*)malloc(sizeof(int16_t) * (size_t)(2 * c->ncoef + 16));
    long* counts = (long*)calloc((size_t)(unsigned)c->ncomp, sizeof(long));
    long nt = 0;
    for (int j = 0; j < c->ncomp; j++) {
        long base;
        const or_subband* s = comp_sb(c, j, &base);
        long start = nt;
        if (type == 0 && s->kind == 0) {
            for (long e = 0; e < (long)s->h * s->w; e++) tok[nt++] = r[base + s->off + e];
        } else {
            for (int a = 0; a < s->h; a++) nt += or_rle_row(r + base + s->off + (long)a * s->w, s->w, tok + nt);
        }
        counts[j] = nt - start;
    }
    need += 2 * nt;
    if (type == 2) need += 2 * nmv;   /* the motion vectors follow the tokens */
    *out_len = need;
    if (frame_type) *frame_type = type;
    if (need > cap) { free(q); free(r); free(tok); free(counts); free(mv); free(pred); return OR_ECAPACITY; }
    memset(out, 0, 32);
    out[0] = 'C'; out[1] = 'V'; out[2] = 'C'; out[3] = '1';
    out[4] = 1;
    out[5] = (uint8_t)flags_byte(c);
    out[6] = (uint8_t)type;
    out[7] = (uint8_t)c->L;
    put32(out + 8, (unsigned long)c->enc_frame);
    put16(out + 12, (unsigned)c->Ho);
    put16(out + 14, (unsigned)c->Wo);
    for (int j = 0; j < c->L; j++) out[16 + j] = (uint8_t)c->k[j];
    put16(out + 22, (unsigned)c->qph);
    put16(out + 24, (unsigned)c->qpl);
    put32(out + 28, (unsigned long)c->ncomp);
    for (int j = 0; j < c->ncomp; j++) put32(out + 32 + 4 * j, (unsigned long)counts[j]);
    uint8_t* tp = out + 32 + 4 * c->ncomp;
    for (long i = 0; i < nt; i++) put16(tp + 2 * i, (unsigned)(uint16_t)tok[i]);
    if (type == 2) memcpy(tp + 2 * nt, mv, (size_t)(2 * nmv));
    memcpy(c->enc_state, q, sizeof(int16_t) * (size_t)c->ncoef);
    if (c->range) memcpy(c->enc_luma, luma, (size_t)c->Hp * c->Wp);
    c->enc_frame += 1;
    free(q); free(r); free(tok); free(counts); free(mv); free(pred);
    return OR_OK;
}

int or_encode(or_codec* c, const uint8_t* rgb, uint8_t* out, long cap, long* out_len,
              int* frame_type, double* coeffs_out) {
    long ny = (long)c->Hp * c->Wp, nc = (long)c->Hcp * c->Wcp;
    double* pl = (double*)malloc(sizeof(double) * (size_t)(ny + 2 * nc));
    double* co = (double*)malloc(sizeof(double) * (size_t)c->ncoef);
    or_codec_planes(c, rgb, pl, pl + ny, pl + ny + nc);
    or_ct_taps(0, pl, c->Hp, c->Wp, c->L, c->k, c->taps, co);
    or_ct_taps(0, pl + ny, c->Hcp, c->Wcp, c->L, c->k, c->taps, co + c->ly.total);
    or_ct_taps(0, pl + ny + nc, c->Hcp, c->Wcp, c->L, c->k, c->taps, co + c->ly.total + c->lc.total);
    float* cf = (float*)malloc(sizeof(float) * (size_t)c->ncoef);
    for (long i = 0; i < c->ncoef; i++) cf[i] = (float)co[i];
    if (coeffs_out) memcpy(coeffs_out, co, sizeof(double) * (size_t)c->ncoef);
    /* the padded luma plane holds integers in [0, 255] */
    uint8_t* luma = (uint8_t*)malloc((size_t)ny);
    for (long i = 0; i < ny; i++) luma[i] = (uint8_t)pl[i];
    int st = or_encode_from_coeffs_luma(c, cf, luma, out, cap, out_len, frame_type);
    free(pl); free(co); free(cf); free(luma);
    return st;
}

/* §3.9 / decoding: undo RLE, undo the frame-type differencing, dequantise
 * (lowpass also rescaled by 2^L), inverse CT, crop the padding, round (ties
 * away from zero, single precision) and clamp: Y to [0,255], Co/Cg to
 * [-255,255]; upsample the chroma and invert the colour transform.          */
int or_decode(or_codec* c, const uint8_t* in, long len, uint8_t* rgb, double* planes_out) {
    return or_decode_scaled(c, in, len, 0, rgb, planes_out);
}

/* the same at scale s in [0, L] (§3.3; see oracle.h) */
int or_decode_scaled(or_codec* c, const uint8_t* in, long len, int scale, uint8_t* rgb, double* planes_out) {
    if (scale < 0 || scale > c->L) return OR_EINVAL;
    if (len < 32 || in[0] != 'C' || in[1] != 'V' || in[2] != 'C' || in[3] != '1') return OR_ECORRUPT;
    if (in[4] != 1 || in[5] != flags_byte(c)) return OR_ECORRUPT;
    int type = in[6];
    if (type > 2 || (type == 2 && !c->range) || in[7] != c->L || get16(in + 12) != (unsigned)c->Ho || get16(in + 14) != (unsigned)c->Wo)
        return OR_ECORRUPT;
    for (int j = 0; j < c->L; j++) if (in[16 + j] != c->k[j]) return OR_ECORRUPT;
    if (get16(in + 22) != (unsigned)c->qph || get16(in + 24) != (unsigned)c->qpl) return OR_ECORRUPT;
    if (get32(in + 28) != (unsigned long)c->ncomp) return OR_ECORRUPT;
    long fidx = (long)get32(in + 8);
    if (type >= 1 && fidx != c->dec_next) return OR_ESTATE;
    /* §3.3: a stream may arrive without its finest `drop` levels; it then serves
     * scales >= drop only, and a P-frame needs the state of levels > scale */
    int drop = (int)get16(in + 26);
    if (drop > c->L) return OR_ECORRUPT;
    if (drop > scale || (type >= 1 && c->dec_floor > scale)) return OR_ESTATE;
    if (len < 32 + 4L * c->ncomp) return OR_ECORRUPT;
    long nt = 0;
    for (int j = 0; j < c->ncomp; j++) nt += (long)get32(in + 32 + 4 * j);
    long nmv = type == 2 ? (long)c->nby * c->nbx : 0;
    if (32 + 4L * c->ncomp + 2 * nt + 2 * nmv > len) return OR_ECORRUPT;
    const uint8_t* tp = in + 32 + 4 * c->ncomp;
    const int8_t* mv = (const int8_t*)(tp + 2 * nt);
    for (long b = 0; b < 2 * nmv; b++)
        if (mv[b] < -c->range || mv[b] > c->range) return OR_ECORRUPT;
    int16_t* r = (int16_t*)malloc(sizeof(int16_t) * (size_t)c->ncoef);
    int16_t* q = (int16_t*)malloc(sizeof(int16_t) * (size_t)c->ncoef);
    long t0 = 0;
    int st = OR_OK;
    for (int j = 0; j < c->ncomp && st == OR_OK; j++) {
        long base, cnt = (long)get32(in + 32 + 4 * j);
        const or_subband* s = comp_sb(c, j, &base);
        long n = (long)s->h * s->w;
        int16_t* tk = (int16_t*)malloc(sizeof(int16_t) * (size_t)(cnt + 1));
        for (long i = 0; i < cnt; i++) tk[i] = (int16_t)get16(tp + 2 * (t0 + i));
        if (s->kind != 0 && s->level <= drop) {
            /* dropped component: no tokens; its residual is zero */
            if (cnt != 0) st = OR_ECORRUPT;
            else memset(r + base + s->off, 0, sizeof(int16_t) * (size_t)n);
        } else if (type == 0 && s->kind == 0) {
            if (cnt != n) st = OR_ECORRUPT;
            else memcpy(r + base + s->off, tk, sizeof(int16_t) * (size_t)n);
        } else {
            st = or_rle_expand(tk, cnt, r + base + s->off, n);
        }
        free(tk);
        t0 += cnt;
    }
    if (st) { free(r); free(q); return st; }
    int16_t* pred = NULL;
    if (type == 2) {
        pred = (int16_t*)malloc(sizeof(int16_t) * (size_t)c->ncoef);
        for (int j = 0; j < c->ncomp; j++) mc_predict(c, j, c->dec_state, mv, pred);
    }
    for (int j = 0; j < c->ncomp; j++) {
        long base;
        const or_subband* s = comp_sb(c, j, &base);
        for (int a = 0; a < s->h; a++)
            for (int b = 0; b < s->w; b++) {
                long idx = base + s->off + (long)a * s->w + b;
                int v;
                if (type == 2) v = r[idx] + pred[idx];
                else if (type == 1) v = r[idx] + c->dec_state[idx];
                else if (s->kind == 0 && a > 0) v = r[idx] + q[idx - s->w];
                else v = r[idx];
                q[idx] = (int16_t)(uint16_t)(v & 0xFFFF);
            }
    }
    free(pred);
    double* co = (double*)malloc(sizeof(double) * (size_t)c->ncoef);
    for (int j = 0; j < c->ncomp; j++) {
        long base;
        const or_subband* s = comp_sb(c, j, &base);
        double scale = s->kind == 0 ? ldexp((double)c->qpl, c->L) : (double)c->qph;
        for (long e = 0; e < (long)s->h * s->w; e++) co[base + s->off + e] = q[base + s->off + e] * scale;
    }
    /* §3.3 scalability: scale s keeps the lowpass and levels s+1..L, which form the
     * sub-pyramid of the (Hp >> s) x (Wp >> s) level-s lowpass image; its inverse is
     * c_s, normalised by the DC gain 2^-s of s levels. */
    const int s = scale;
    const int Hps = c->Hp >> s, Wps = c->Wp >> s, Hcps = c->Hcp >> s, Wcps = c->Wcp >> s;
    const int Hos = (c->Ho + (1 << s) - 1) >> s, Wos = (c->Wo + (1 << s) - 1) >> s;
    const int Hcs = (c->Hc + (1 << s) - 1) >> s, Wcs = (c->Wc + (1 << s) - 1) >> s;
    long ny = (long)Hps * Wps, nc = (long)Hcps * Wcps;
    double* pl = (double*)malloc(sizeof(double) * (size_t)(ny + 2 * nc));
    const or_layout* lays[3] = {&c->ly, &c->lc, &c->lc};
    const long poff[3] = {0, c->ly.total, c->ly.total + c->lc.total};
    const long ploff[3] = {0, ny, ny + nc};
    const int ph[3] = {Hps, Hcps, Hcps}, pw[3] = {Wps, Wcps, Wcps};
    for (int p = 0; p < 3; p++) {
        const or_layout* ly = lays[p];
        const double* cp = co + poff[p];
        long nlow = (long)ly->sb[0].h * ly->sb[0].w;
        if (s == c->L) {
            memcpy(pl + ploff[p], cp, sizeof(double) * (size_t)nlow);
        } else {
            /* first subband of level s+1 */
            int first = 1;
            for (int j = 0; j < s; j++) first += 1 << c->k[j];
            long tail = ly->total - ly->sb[first].off;
            double* sub = (double*)malloc(sizeof(double) * (size_t)(nlow + tail));
            memcpy(sub, cp, sizeof(double) * (size_t)nlow);
            memcpy(sub + nlow, cp + ly->sb[first].off, sizeof(double) * (size_t)tail);
            or_ct_taps(1, sub, ph[p], pw[p], c->L - s, c->k + s, c->taps, pl + ploff[p]);
            free(sub);
        }
        for (long e = 0; e < (long)ph[p] * pw[p]; e++) pl[ploff[p] + e] = ldexp(pl[ploff[p] + e], -s);
    }
    if (planes_out) memcpy(planes_out, pl, sizeof(double) * (size_t)(ny + 2 * nc));
    long n = (long)Hos * Wos, ncs = (long)Hcs * Wcs;
    int16_t* Y = (int16_t*)malloc(sizeof(int16_t) * n);
    int16_t* Co = (int16_t*)malloc(sizeof(int16_t) * n);
    int16_t* Cg = (int16_t*)malloc(sizeof(int16_t) * n);
    int16_t* Co2 = (int16_t*)malloc(sizeof(int16_t) * ncs);
    int16_t* Cg2 = (int16_t*)malloc(sizeof(int16_t) * ncs);
    /* chroma: YCoCg-R values in [-255, 255], or bytes offset by 127 under 8-bit storage */
    const int clo = c->st8 ? 0 : -255;
    for (int y = 0; y < Hos; y++)
        for (int x = 0; x < Wos; x++)
            Y[(long)y * Wos + x] = (int16_t)clampi((long)roundf((float)pl[(long)y * Wps + x]), 0, 255);
    for (int y = 0; y < Hcs; y++)
        for (int x = 0; x < Wcs; x++) {
            Co2[(long)y * Wcs + x] = (int16_t)clampi((long)roundf((float)pl[ny + (long)y * Wcps + x]), clo, 255);
            Cg2[(long)y * Wcs + x] = (int16_t)clampi((long)roundf((float)pl[ny + nc + (long)y * Wcps + x]), clo, 255);
        }
    or_chroma_up(Co2, Hcs, Wcs, Hos, Wos, Co);
    or_chroma_up(Cg2, Hcs, Wcs, Hos, Wos, Cg);
    if (c->st8) or_ycocg8_inverse(Y, Co, Cg, n, rgb);
    else or_ycocgr_inverse(Y, Co, Cg, n, rgb);
    memcpy(c->dec_state, q, sizeof(int16_t) * (size_t)c->ncoef);
    c->dec_next = fidx + 1;
    c->dec_floor = type == 0 ? drop : (drop > c->dec_floor ? drop : c->dec_floor);
    free(r); free(q); free(co); free(pl); free(Y); free(Co); free(Cg); free(Co2); free(Cg2);
    return OR_OK;
}

/* §3.3, §3.9: a receiver that wants scale s needs only the lowpass and levels
 * s+1..L, so the finest `drop` levels can be left out of a frame without
 * re-encoding: their token counts become 0, their tokens go, and header bytes
 * 26-27 record `drop`.  A stream already missing d0 levels can only lose more. */
int or_stream_drop(const or_codec* c, const uint8_t* in, long len, int drop, uint8_t* out, long cap,
                   long* out_len) {
    if (len < 32 || in[0] != 'C' || in[1] != 'V' || in[2] != 'C' || in[3] != '1') return OR_ECORRUPT;
    if (in[7] != c->L || get32(in + 28) != (unsigned long)c->ncomp) return OR_ECORRUPT;
    if (len < 32 + 4L * c->ncomp) return OR_ECORRUPT;
    int d0 = (int)get16(in + 26);
    if (drop < d0 || drop > c->L) return OR_EINVAL;
    long ntot = 0, nkeep = 0;
    for (int j = 0; j < c->ncomp; j++) {
        long base, cnt = (long)get32(in + 32 + 4 * j);
        const or_subband* s = comp_sb(c, j, &base);
        ntot += cnt;
        if (!(s->kind != 0 && s->level <= drop)) nkeep += cnt;
    }
    long hdr = 32 + 4L * c->ncomp;
    if (hdr + 2 * ntot > len) return OR_ECORRUPT;
    long tail = len - (hdr + 2 * ntot);   /* the motion vectors of a P-frame with motion */
    *out_len = hdr + 2 * nkeep + tail;
    if (*out_len > cap) return OR_ECAPACITY;
    memcpy(out, in, 32);
    put16(out + 26, (unsigned)drop);
    long src = hdr, dst = hdr;
    for (int j = 0; j < c->ncomp; j++) {
        long base, cnt = (long)get32(in + 32 + 4 * j);
        const or_subband* s = comp_sb(c, j, &base);
        int keep = !(s->kind != 0 && s->level <= drop);
        put32(out + 32 + 4 * j, keep ? (unsigned long)cnt : 0UL);
        if (keep) {
            memcpy(out + dst, in + src, (size_t)(2 * cnt));
            dst += 2 * cnt;
        }
        src += 2 * cnt;
    }
    memcpy(out + dst, in + src, (size_t)tail);
    return OR_OK;
}

/* ---------------------------------------------------------------- DEFLATE */
/* cost (sum of frequency x code length) of an optimal prefix code: the sum of
 * the weights of the internal nodes Huffman's pairing creates (§3.9's DEFLATE
 * codes are Huffman codes); *depth receives the longest code length */
unsigned long long or_huffman_cost(const unsigned long* freq, int n, int* depth) {
    unsigned long long w[2 * 300];
    int dep[2 * 300], alive[2 * 300], m = 0;
    for (int i = 0; i < n; i++)
        if (freq[i]) { w[m] = freq[i]; dep[m] = 0; alive[m] = 1; m++; }
    *depth = m == 1 ? 1 : 0;
    if (m < 2) return m == 1 ? (unsigned long long)w[0] : 0;
    /* leaves under each node: track the deepest leaf below every node */
    unsigned long long cost = 0;
    int left = m;
    while (left > 1) {
        int a = -1, b = -1;
        for (int i = 0; i < m; i++) {
            if (!alive[i]) continue;
            if (a < 0 || w[i] < w[a]) { b = a; a = i; }
            else if (b < 0 || w[i] < w[b]) b = i;
        }
        alive[a] = alive[b] = 0;
        w[m] = w[a] + w[b];
        dep[m] = (dep[a] > dep[b] ? dep[a] : dep[b]) + 1;
        alive[m] = 1;
        cost += w[m];
        m++;
        left--;
    }
    *depth = dep[m - 1];
    return cost;
}

static unsigned long rd32u(const uint8_t* p) { return get32(p); }

/* inflate a deflated frame (the container of cvc_deflate_frame) with zlib,
 * each component's raw DEFLATE stream on its own; the segment table is only
 * checked for its size */
int or_inflate_container(const or_codec* c, const uint8_t* in, long len, uint8_t* out, long cap, long* out_len) {
    long hdr = 32 + 4L * c->ncomp;
    if (len < hdr || in[0] != 'C' || in[1] != 'V' || in[2] != 'C' || in[3] != '1' || (in[4] != 2 && in[4] != 3) ||
        in[5] != flags_byte(c) || get32(in + 28) != (unsigned long)c->ncomp)
        return OR_ECORRUPT;
    /* version 2: a stream per component; 3 (CVC-NTS): one stream of all token bytes */
    int nstr = in[4] == 3 ? 1 : c->ncomp;
    if (len < hdr + 4L * nstr) return OR_ECORRUPT;
    long ntok = 0, nseg = 0;
    for (int j = 0; j < c->ncomp; j++) {
        long n = (long)rd32u(in + 32 + 4 * j);
        ntok += n;
        nseg += (2 * n + 255) / 256;
    }
    if (nstr == 1) nseg = (2 * ntok + 255) / 256;
    long mvb = in[6] == 2 ? 2L * ((c->Hp + 15) / 16) * ((c->Wp + 15) / 16) : 0;
    *out_len = hdr + 2 * ntok + mvb;
    if (*out_len > cap) return OR_ECAPACITY;
    long pos = hdr + 4L * nstr + ((2 * nseg + 3) & ~3L);
    memcpy(out, in, (size_t)hdr);
    out[4] = 1;
    long o = hdr;
    for (int j = 0; j < nstr; j++) {
        long n = nstr == 1 ? ntok : (long)rd32u(in + 32 + 4 * j), nb = (long)rd32u(in + hdr + 4 * j);
        if ((n == 0) != (nb == 0) || pos + nb > len) return OR_ECORRUPT;
        if (n) {
            z_stream z;
            memset(&z, 0, sizeof(z));
            if (inflateInit2(&z, -15) != Z_OK) return OR_ECORRUPT;
            z.next_in = (Bytef*)(in + pos);
            z.avail_in = (uInt)nb;
            z.next_out = out + o;
            z.avail_out = (uInt)(2 * n);
            int r = inflate(&z, Z_FINISH);
            long got = (long)(2 * n) - (long)z.avail_out;
            inflateEnd(&z);
            if (r != Z_STREAM_END || got != 2 * n) return OR_ECORRUPT;
        }
        pos += nb;
        o += 2 * n;
    }
    if (pos + mvb > len) return OR_ECORRUPT;
    memcpy(out + o, in + pos, (size_t)mvb);
    return OR_OK;
}

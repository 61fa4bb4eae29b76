/*
 * FP64 CPU oracle of the learned orientation proposal: a small convolutional
 * network that maps a 128 x 128 pattern to k candidate orientations, each
 * from a 6-D rotation representation made orthonormal by Gram-Schmidt, with a
 * winner-takes-all loss that is invariant under the 24 proper rotations of
 * the cubic point group.
 *
 * TEST INFRASTRUCTURE ONLY (used by the tests and nothing else; shares no
 * code with the CUDA library).  The paper indexes by template matching only;
 * this proposal network is an extension of it whose architecture is a stated
 * reading:
 *   input   x [128, 128], standardised per pattern (zero mean, unit std, as the
 *           paper's pre-processing does before correlation, Section 2.2)
 *   conv l  3 x 3, stride 2, zero padding 1, bias, ReLU, channels
 *           1 -> 32 -> 64 -> 64 -> 128 -> 128 (sides 64, 32, 16, 8, 4)
 *   pool    mean over the 4 x 4 positions -> 128
 *   fc1     128 -> 256, ReLU
 *   fc2     256 -> 6k  (k heads, 6 numbers each)
 *   head h  a1 = out[6h..6h+2], a2 = out[6h+3..6h+5] -> R = [b1 b2 b3]
 *           b1 = a1/|a1|, b2 = normalised (a2 - (b1.a2) b1), b3 = b1 x b2
 *   loss    min over heads h and cubic operators S of |R_h - S R_gt|_F^2,
 *           averaged over the batch; R_gt = R(q_gt), the projector's matrix of
 *           the ground-truth orientation.
 * Parameters are one flat float array in the order conv1 W, b, ..., conv5 W,
 * b, fc1 W, b, fc2 W, b; conv W[co][ci][ky][kx], fc W[out][in].
 * The optimiser is Adam (Kingma & Ba 2015) with bias correction.
 *
 * The architecture is a reading (the paper has no network); every function
 * below is pinned by library routines, finite differences or closed forms in
 * tests/test_oracle_cnn.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define CNN_SIDE 128
#define CNN_LAYERS 5
static const int kCh[CNN_LAYERS + 1] = {1, 32, 64, 64, 128, 128};
#define CNN_FC1 256

/* ------------------------------------------------------------ parameters */
static long conv_w_count(int l) { return (long)kCh[l + 1] * kCh[l] * 9; }

/* offsets of every parameter block in the flat array; returns the total */
static long param_offsets(int k, long conv_w[CNN_LAYERS], long conv_b[CNN_LAYERS], long *fc1_w, long *fc1_b,
                          long *fc2_w, long *fc2_b) {
    long o = 0;
    for (int l = 0; l < CNN_LAYERS; ++l) {
        conv_w[l] = o;
        o += conv_w_count(l);
        conv_b[l] = o;
        o += kCh[l + 1];
    }
    *fc1_w = o;
    o += (long)CNN_FC1 * kCh[CNN_LAYERS];
    *fc1_b = o;
    o += CNN_FC1;
    *fc2_w = o;
    o += (long)6 * k * CNN_FC1;
    *fc2_b = o;
    o += 6 * k;
    return o;
}

long orc_cnn_num_params(int k) {
    long a[CNN_LAYERS], b[CNN_LAYERS], c, d, e, f;
    return param_offsets(k, a, b, &c, &d, &e, &f);
}

/* ---------------------------------------------------------------- layers */
/* per-pattern standardisation: (x - mean) / std, population std; a constant
 * image becomes all zeros */
void orc_cnn_standardise(const double *x, int n, double *y) {
    double s = 0.0, s2 = 0.0;
    for (int i = 0; i < n; ++i) s += x[i];
    const double mean = s / n;
    for (int i = 0; i < n; ++i) s2 += (x[i] - mean) * (x[i] - mean);
    const double sd = sqrt(s2 / n);
    const int degenerate = !(sd > 1e-12 * (1.0 + fabs(mean)));
    for (int i = 0; i < n; ++i) y[i] = degenerate ? 0.0 : (x[i] - mean) / sd;
}

/* y[co][oy][ox] = b[co] + sum_ci sum_ky,kx w[co][ci][ky][kx] x[ci][2oy-1+ky][2ox-1+kx]
 * (zero outside), input side s, output side s/2; no activation */
void orc_conv3x3s2(const double *x, int ci_n, int s, const double *w, const double *b, int co_n, double *y) {
    const int so = s / 2;
    for (int co = 0; co < co_n; ++co)
        for (int oy = 0; oy < so; ++oy)
            for (int ox = 0; ox < so; ++ox) {
                double acc = b ? b[co] : 0.0;
                for (int ci = 0; ci < ci_n; ++ci)
                    for (int ky = 0; ky < 3; ++ky) {
                        const int iy = 2 * oy - 1 + ky;
                        if (iy < 0 || iy >= s) continue;
                        for (int kx = 0; kx < 3; ++kx) {
                            const int ix = 2 * ox - 1 + kx;
                            if (ix < 0 || ix >= s) continue;
                            acc += w[((long)co * ci_n + ci) * 9 + ky * 3 + kx] * x[((long)ci * s + iy) * s + ix];
                        }
                    }
                y[((long)co * so + oy) * so + ox] = acc;
            }
}

/* Gram-Schmidt of the 6-D representation: R (row-major 3 x 3) has columns
 * b1, b2, b3 (Zhou, Barnes, Lu, Yang & Li 2019, Section 4.2) */
static void cross3(const double a[3], const double b[3], double c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

void orc_gram_schmidt(const double a[6], double R[9]) {
    double b1[3], b2[3], b3[3], u[3];
    const double n1 = sqrt(dot3(a, a));
    for (int i = 0; i < 3; ++i) b1[i] = a[i] / n1;
    const double d = dot3(b1, a + 3);
    for (int i = 0; i < 3; ++i) u[i] = a[3 + i] - d * b1[i];
    const double n2 = sqrt(dot3(u, u));
    for (int i = 0; i < 3; ++i) b2[i] = u[i] / n2;
    cross3(b1, b2, b3);
    for (int i = 0; i < 3; ++i) {
        R[i * 3 + 0] = b1[i];
        R[i * 3 + 1] = b2[i];
        R[i * 3 + 2] = b3[i];
    }
}

/* gradient of a scalar through Gram-Schmidt: G = dL/dR (row-major) -> ga = dL/da */
void orc_gram_schmidt_backward(const double a[6], const double G[9], double ga[6]) {
    double b1[3], b2[3], u[3], g1[3], g2[3], g3[3], gb1[3], gb2[3], gu[3], t[3];
    const double n1 = sqrt(dot3(a, a));
    for (int i = 0; i < 3; ++i) b1[i] = a[i] / n1;
    const double d = dot3(b1, a + 3);
    for (int i = 0; i < 3; ++i) u[i] = a[3 + i] - d * b1[i];
    const double n2 = sqrt(dot3(u, u));
    for (int i = 0; i < 3; ++i) b2[i] = u[i] / n2;
    for (int i = 0; i < 3; ++i) {
        g1[i] = G[i * 3 + 0];
        g2[i] = G[i * 3 + 1];
        g3[i] = G[i * 3 + 2];
    }
    /* b3 = b1 x b2: d(b3).g3 = db1.(b2 x g3) + db2.(g3 x b1) */
    cross3(b2, g3, t);
    for (int i = 0; i < 3; ++i) gb1[i] = g1[i] + t[i];
    cross3(g3, b1, t);
    for (int i = 0; i < 3; ++i) gb2[i] = g2[i] + t[i];
    /* b2 = u / |u| */
    const double pb2 = dot3(b2, gb2);
    for (int i = 0; i < 3; ++i) gu[i] = (gb2[i] - pb2 * b2[i]) / n2;
    /* u = a2 - (b1.a2) b1 */
    const double pu = dot3(b1, gu);
    for (int i = 0; i < 3; ++i) {
        ga[3 + i] = gu[i] - pu * b1[i];
        gb1[i] += -pu * a[3 + i] - d * gu[i];
    }
    /* b1 = a1 / |a1| */
    const double pb1 = dot3(b1, gb1);
    for (int i = 0; i < 3; ++i) ga[i] = (gb1[i] - pb1 * b1[i]) / n1;
}

/* rotation matrix of a unit quaternion: the projector's own (xcf_oracle.c) */
void orc_quat_to_matrix(const double q[4], double R[9]);
static void quat_to_R(const double q[4], double R[9]) { orc_quat_to_matrix(q, R); }

/* the 24 proper rotations of the cubic group as signed permutation matrices
 * with determinant +1 (enumerated, not tabulated) */
static int cubic_matrices(double S[24][9]) {
    static const int perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    int n = 0;
    for (int p = 0; p < 6; ++p)
        for (int s = 0; s < 8; ++s) {
            double M[9] = {0};
            for (int r = 0; r < 3; ++r) M[r * 3 + perm[p][r]] = (s >> r & 1) ? -1.0 : 1.0;
            const double det = M[0] * (M[4] * M[8] - M[5] * M[7]) - M[1] * (M[3] * M[8] - M[5] * M[6]) +
                               M[2] * (M[3] * M[7] - M[4] * M[6]);
            if (det > 0) memcpy(S[n++], M, sizeof M);
        }
    return n;
}

void orc_cubic_matrices(double *out /* [24][9] */) {
    double S[24][9];
    cubic_matrices(S);
    memcpy(out, S, sizeof S);
}

/* winner-takes-all loss of one pattern: out6 [6k] -> loss, dL/dout6 (nullable),
 * the winning head and operator; ties go to the lowest (head, operator) */
double orc_cnn_head_loss(const double *out6, int k, const double q_gt[4], double *gout6, int *win_h, int *win_s) {
    double S[24][9], Rg[9], best = INFINITY;
    cubic_matrices(S);
    quat_to_R(q_gt, Rg);
    int bh = 0, bs = 0;
    double bestT[9] = {0};
    for (int h = 0; h < k; ++h) {
        double R[9];
        orc_gram_schmidt(out6 + 6 * h, R);
        for (int s = 0; s < 24; ++s) {
            double T[9], l = 0.0;   /* T = S Rg */
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    double acc = 0.0;
                    for (int m = 0; m < 3; ++m) acc += S[s][i * 3 + m] * Rg[m * 3 + j];
                    T[i * 3 + j] = acc;
                }
            for (int i = 0; i < 9; ++i) l += (R[i] - T[i]) * (R[i] - T[i]);
            if (l < best) {
                best = l;
                bh = h;
                bs = s;
                memcpy(bestT, T, sizeof T);
            }
        }
    }
    if (gout6) {
        memset(gout6, 0, sizeof(double) * 6 * k);
        double R[9], G[9];
        orc_gram_schmidt(out6 + 6 * bh, R);
        for (int i = 0; i < 9; ++i) G[i] = 2.0 * (R[i] - bestT[i]);
        orc_gram_schmidt_backward(out6 + 6 * bh, G, gout6 + 6 * bh);
    }
    if (win_h) *win_h = bh;
    if (win_s) *win_s = bs;
    return best;
}

/* ------------------------------------------------------------- the network */
typedef struct {
    double *x0;                   /* standardised input [128*128]               */
    double *a[CNN_LAYERS];        /* post-ReLU conv outputs                     */
    double pool[128], h1[CNN_FC1];
} acts_t;

static void acts_alloc(acts_t *A) {
    A->x0 = malloc(sizeof(double) * CNN_SIDE * CNN_SIDE);
    int s = CNN_SIDE;
    for (int l = 0; l < CNN_LAYERS; ++l) {
        s /= 2;
        A->a[l] = malloc(sizeof(double) * kCh[l + 1] * s * s);
    }
}
static void acts_free(acts_t *A) {
    free(A->x0);
    for (int l = 0; l < CNN_LAYERS; ++l) free(A->a[l]);
}

double orc_bf16_round(double x);

/* bf16 != 0: the inference form whose convolutions after the first take
 * BF16 operands (the layer input rounded through FP32 to BF16, and the
 * layer's weights likewise); accumulation, bias, ReLU, pool and the fully
 * connected layers unchanged. */
static void forward_one_p(const float *params, const double *x, int k, acts_t *A, double *out, int bf16) {
    long cw[CNN_LAYERS], cb[CNN_LAYERS], f1w, f1b, f2w, f2b;
    const long np = param_offsets(k, cw, cb, &f1w, &f1b, &f2w, &f2b);
    double *p = malloc(sizeof(double) * np);
    for (long i = 0; i < np; ++i) p[i] = params[i];
    orc_cnn_standardise(x, CNN_SIDE * CNN_SIDE, A->x0);
    const double *in = A->x0;
    int s = CNN_SIDE;
    for (int l = 0; l < CNN_LAYERS; ++l) {
        if (bf16 && l > 0) {
            const long nin = (long)kCh[l] * s * s;
            for (long i = 0; i < nin; ++i) A->a[l - 1][i] = orc_bf16_round(A->a[l - 1][i]);
            for (long i = 0; i < conv_w_count(l); ++i) p[cw[l] + i] = orc_bf16_round(p[cw[l] + i]);
        }
        orc_conv3x3s2(in, kCh[l], s, p + cw[l], p + cb[l], kCh[l + 1], A->a[l]);
        s /= 2;
        const long cnt = (long)kCh[l + 1] * s * s;
        for (long i = 0; i < cnt; ++i) A->a[l][i] = A->a[l][i] > 0.0 ? A->a[l][i] : 0.0;
        in = A->a[l];
    }
    const int C5 = kCh[CNN_LAYERS];
    for (int c = 0; c < C5; ++c) {
        double acc = 0.0;
        for (int i = 0; i < s * s; ++i) acc += in[c * s * s + i];
        A->pool[c] = acc / (s * s);
    }
    for (int o = 0; o < CNN_FC1; ++o) {
        double acc = p[f1b + o];
        for (int i = 0; i < C5; ++i) acc += p[f1w + (long)o * C5 + i] * A->pool[i];
        A->h1[o] = acc > 0.0 ? acc : 0.0;
    }
    for (int o = 0; o < 6 * k; ++o) {
        double acc = p[f2b + o];
        for (int i = 0; i < CNN_FC1; ++i) acc += p[f2w + (long)o * CNN_FC1 + i] * A->h1[i];
        out[o] = acc;
    }
    free(p);
}

static void forward_one(const float *params, const double *x, int k, acts_t *A, double *out) {
    forward_one_p(params, x, k, A, out, 0);
}

/* out [B][6k] for images x [B][128][128] */
void orc_cnn_forward(const float *params, const double *x, int B, int k, double *out) {
#pragma omp parallel for schedule(dynamic)
    for (int b = 0; b < B; ++b) {
        acts_t A;
        acts_alloc(&A);
        forward_one(params, x + (long)b * CNN_SIDE * CNN_SIDE, k, &A, out + (long)b * 6 * k);
        acts_free(&A);
    }
}

/* the BF16 inference form of orc_cnn_forward (see forward_one_p) */
void orc_cnn_forward_bf16(const float *params, const double *x, int B, int k, double *out) {
#pragma omp parallel for schedule(dynamic)
    for (int b = 0; b < B; ++b) {
        acts_t A;
        acts_alloc(&A);
        forward_one_p(params, x + (long)b * CNN_SIDE * CNN_SIDE, k, &A, out + (long)b * 6 * k, 1);
        acts_free(&A);
    }
}

/* mean loss over the batch and its gradient with respect to every parameter
 * (grad [n_params], summed over patterns then divided by B); winners [B][2]
 * (head, operator) nullable */
double orc_cnn_loss_grad(const float *params, const double *x, int B, int k, const double *q_gt, double *grad,
                         int *winners) {
    long cw[CNN_LAYERS], cb[CNN_LAYERS], f1w, f1b, f2w, f2b;
    const long np = param_offsets(k, cw, cb, &f1w, &f1b, &f2w, &f2b);
    double *p = malloc(sizeof(double) * np);
    for (long i = 0; i < np; ++i) p[i] = params[i];
    if (grad) memset(grad, 0, sizeof(double) * np);
    double loss_sum = 0.0;
    const int C5 = kCh[CNN_LAYERS];
    for (int b = 0; b < B; ++b) {   /* sequential: the gradient sum has one order */
        acts_t A;
        acts_alloc(&A);
        double *out = malloc(sizeof(double) * 6 * k), *gout = malloc(sizeof(double) * 6 * k);
        forward_one(params, x + (long)b * CNN_SIDE * CNN_SIDE, k, &A, out);
        int wh, ws;
        loss_sum += orc_cnn_head_loss(out, k, q_gt + 4 * b, gout, &wh, &ws);
        if (winners) {
            winners[2 * b] = wh;
            winners[2 * b + 1] = ws;
        }
        if (grad) {
            const double inv_b = 1.0 / B;
            double gh1[CNN_FC1], gpool[128];
            for (int o = 0; o < 6 * k; ++o) gout[o] *= inv_b;
            /* fc2 */
            for (int i = 0; i < CNN_FC1; ++i) gh1[i] = 0.0;
            for (int o = 0; o < 6 * k; ++o) {
                grad[f2b + o] += gout[o];
                for (int i = 0; i < CNN_FC1; ++i) {
                    grad[f2w + (long)o * CNN_FC1 + i] += gout[o] * A.h1[i];
                    gh1[i] += gout[o] * p[f2w + (long)o * CNN_FC1 + i];
                }
            }
            /* ReLU of fc1 */
            for (int i = 0; i < CNN_FC1; ++i)
                if (!(A.h1[i] > 0.0)) gh1[i] = 0.0;
            for (int i = 0; i < C5; ++i) gpool[i] = 0.0;
            for (int o = 0; o < CNN_FC1; ++o) {
                grad[f1b + o] += gh1[o];
                for (int i = 0; i < C5; ++i) {
                    grad[f1w + (long)o * C5 + i] += gh1[o] * A.pool[i];
                    gpool[i] += gh1[o] * p[f1w + (long)o * C5 + i];
                }
            }
            /* mean pool of conv5 (side 4) */
            int s = CNN_SIDE >> CNN_LAYERS;
            double *gy = malloc(sizeof(double) * C5 * s * s);
            for (int c = 0; c < C5; ++c)
                for (int i = 0; i < s * s; ++i) gy[c * s * s + i] = gpool[c] / (s * s);
            /* conv layers, last to first: gy is dL/d(post-ReLU output) */
            for (int l = CNN_LAYERS - 1; l >= 0; --l) {
                const int so = s, si = 2 * s, ci_n = kCh[l], co_n = kCh[l + 1];
                const double *xin = l > 0 ? A.a[l - 1] : A.x0;
                const double *yout = A.a[l];
                double *gx = calloc((size_t)ci_n * si * si, sizeof(double));
                for (int co = 0; co < co_n; ++co)
                    for (int oy = 0; oy < so; ++oy)
                        for (int ox = 0; ox < so; ++ox) {
                            const long oi = ((long)co * so + oy) * so + ox;
                            const double g = yout[oi] > 0.0 ? gy[oi] : 0.0;
                            if (g == 0.0) continue;
                            grad[cb[l] + co] += g;
                            for (int ci = 0; ci < ci_n; ++ci)
                                for (int ky = 0; ky < 3; ++ky) {
                                    const int iy = 2 * oy - 1 + ky;
                                    if (iy < 0 || iy >= si) continue;
                                    for (int kx = 0; kx < 3; ++kx) {
                                        const int ix = 2 * ox - 1 + kx;
                                        if (ix < 0 || ix >= si) continue;
                                        const long wi = ((long)co * ci_n + ci) * 9 + ky * 3 + kx;
                                        const long xi = ((long)ci * si + iy) * si + ix;
                                        grad[cw[l] + wi] += g * xin[xi];
                                        gx[xi] += g * p[cw[l] + wi];
                                    }
                                }
                        }
                free(gy);
                gy = gx;
                s = si;
            }
            free(gy);
        }
        free(out);
        free(gout);
        acts_free(&A);
    }
    free(p);
    return loss_sum / B;
}

/* one Adam step (Kingma & Ba 2015, Algorithm 1), t >= 1 the step number */
void orc_adam(double *params, const double *grad, double *m, double *v, long n, int t, double lr, double b1,
              double b2, double eps) {
    const double c1 = 1.0 - pow(b1, t), c2 = 1.0 - pow(b2, t);
    for (long i = 0; i < n; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * grad[i];
        v[i] = b2 * v[i] + (1.0 - b2) * grad[i] * grad[i];
        params[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
    }
}

/* unit quaternion (w >= 0) of a rotation matrix, from the largest of the four
 * squared components (Shepperd 1978) */
void orc_matrix_to_quat(const double R[9], double q[4]) {
    const double t = R[0] + R[4] + R[8];
    double w, x, y, z;
    const double c[4] = {1 + t, 1 + R[0] - R[4] - R[8], 1 - R[0] + R[4] - R[8], 1 - R[0] - R[4] + R[8]};
    int m = 0;
    for (int i = 1; i < 4; ++i)
        if (c[i] > c[m]) m = i;
    const double s = 2.0 * sqrt(c[m]);
    /* for R(q) of the projector: R[7] - R[5] = 4wx, R[2] - R[6] = 4wy, R[3] - R[1] = 4wz,
     * R[1] + R[3] = 4xy, R[2] + R[6] = 4xz, R[5] + R[7] = 4yz */
    switch (m) {
        case 0: w = s / 4; x = (R[7] - R[5]) / s; y = (R[2] - R[6]) / s; z = (R[3] - R[1]) / s; break;
        case 1: x = s / 4; w = (R[7] - R[5]) / s; y = (R[1] + R[3]) / s; z = (R[2] + R[6]) / s; break;
        case 2: y = s / 4; w = (R[2] - R[6]) / s; x = (R[1] + R[3]) / s; z = (R[5] + R[7]) / s; break;
        default: z = s / 4; w = (R[3] - R[1]) / s; x = (R[2] + R[6]) / s; y = (R[5] + R[7]) / s; break;
    }
    const double nn = sqrt(w * w + x * x + y * y + z * z), sg = w < 0 ? -1.0 : 1.0;
    q[0] = sg * w / nn;
    q[1] = sg * x / nn;
    q[2] = sg * y / nn;
    q[3] = sg * z / nn;
}

/* proposals: out [B][6k] -> quats [B][k][4] */
void orc_cnn_proposals(const double *out, int B, int k, double *quats) {
    for (int b = 0; b < B; ++b)
        for (int h = 0; h < k; ++h) {
            double R[9];
            orc_gram_schmidt(out + ((long)b * k + h) * 6, R);
            orc_matrix_to_quat(R, quats + ((long)b * k + h) * 4);
        }
}

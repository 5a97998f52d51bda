/*
 * FP64 reference of the warm-start network for the tau = 0+ link solve
 * (test infrastructure; see oracle.h).  The paper has no learned component; the
 * network is the one the build trains to predict a starting point for the
 * Newton iteration of the boost-invariant matching condition (ic.c).
 *
 * Starting point U0 = exp(i (delta_s + delta_net)^a t^a) U1 U2, where, with
 * a1 = im_tl(U1), a2 = im_tl(U2) and c = i[a1, a2] (algebra components),
 *   delta_s = -c/2 - (3/8) i[a1, c] - (1/8) i[a2, c]
 * is the small-field series of the solution's offset from U1 U2, exact through
 * third order in the link fields (residual O(a^4); pinned by its scaling in
 * tests/test_oracle_mlp.py), and delta_net is the network's correction:
 *   input  x (36) / x_scale: a1, a2, c, delta_s + c/2, |a1|^2, |a2|^2, a1.a2, |c|^2
 *   h1 = tanh(W1 x + b1)      W1: 128 x 36
 *   h2 = tanh(W2 h1 + b2)     W2: 128 x 128
 *   y  = W3 h2 + b3           W3: 16 x 128   (outputs 0..7: delta_net / y_scale, 8..15: padding)
 *   target: delta - delta_s with delta^a = 2 Im Tr[t^a U (U1 U2)^dag] of the Newton
 *           solution U; outputs 8..15 -> 0
 *   loss = mean over the batch and the 16 outputs of (y - target)^2
 * Pins (tests/test_oracle_mlp.py): backward against central finite differences of
 * the loss; the series against the Newton solution (abelian case exact, O(a^4)
 * residual); the features against the Lie bracket of the Gell-Mann generators.
 */
#include <math.h>
#include <string.h>
#include "oracle.h"

#define NI 36
#define NH 128
#define NO 16

void o_mlp_forward(int batch, const double *x, const double *W1, const double *b1, const double *W2,
                   const double *b2, const double *W3, const double *b3, double *h1, double *h2,
                   double *y) {
    for (int m = 0; m < batch; m++) {
        const double *xm = x + NI * m;
        double *a = h1 + NH * m, *b = h2 + NH * m, *o = y + NO * m;
        for (int j = 0; j < NH; j++) {
            double s = b1[j];
            for (int k = 0; k < NI; k++) s += W1[NI * j + k] * xm[k];
            a[j] = tanh(s);
        }
        for (int j = 0; j < NH; j++) {
            double s = b2[j];
            for (int k = 0; k < NH; k++) s += W2[NH * j + k] * a[k];
            b[j] = tanh(s);
        }
        for (int j = 0; j < NO; j++) {
            double s = b3[j];
            for (int k = 0; k < NH; k++) s += W3[NH * j + k] * b[k];
            o[j] = s;
        }
    }
}

double o_mlp_loss_backward(int batch, const double *x, const double *target, const double *W1,
                           const double *b1, const double *W2, const double *b2, const double *W3,
                           const double *b3, double *gW1, double *gb1, double *gW2, double *gb2,
                           double *gW3, double *gb3) {
    static double h1[NH], h2[NH], y[NO], d3[NO], d2[NH], d1[NH];
    memset(gW1, 0, sizeof(double) * NH * NI);
    memset(gb1, 0, sizeof(double) * NH);
    memset(gW2, 0, sizeof(double) * NH * NH);
    memset(gb2, 0, sizeof(double) * NH);
    memset(gW3, 0, sizeof(double) * NO * NH);
    memset(gb3, 0, sizeof(double) * NO);
    double loss = 0;
    const double norm = 1.0 / ((double)batch * NO);
    for (int m = 0; m < batch; m++) {
        const double *xm = x + NI * m, *tm = target + NO * m;
        o_mlp_forward(1, xm, W1, b1, W2, b2, W3, b3, h1, h2, y);
        for (int j = 0; j < NO; j++) {
            const double e = y[j] - tm[j];
            loss += e * e * norm;
            d3[j] = 2.0 * e * norm;
        }
        for (int j = 0; j < NO; j++) {
            gb3[j] += d3[j];
            for (int k = 0; k < NH; k++) gW3[NH * j + k] += d3[j] * h2[k];
        }
        for (int k = 0; k < NH; k++) {
            double s = 0;
            for (int j = 0; j < NO; j++) s += W3[NH * j + k] * d3[j];
            d2[k] = s * (1.0 - h2[k] * h2[k]);
        }
        for (int j = 0; j < NH; j++) {
            gb2[j] += d2[j];
            for (int k = 0; k < NH; k++) gW2[NH * j + k] += d2[j] * h1[k];
        }
        for (int k = 0; k < NH; k++) {
            double s = 0;
            for (int j = 0; j < NH; j++) s += W2[NH * j + k] * d2[j];
            d1[k] = s * (1.0 - h1[k] * h1[k]);
        }
        for (int j = 0; j < NH; j++) {
            gb1[j] += d1[j];
            for (int k = 0; k < NI; k++) gW1[NI * j + k] += d1[j] * xm[k];
        }
    }
    return loss;
}

/* third-order series of the offset delta of the solution from U1 U2 (header) */
void o_ic_series(const cplx U1[9], const cplx U2[9], double ds[8]) {
    double a1[8], a2[8], c[8], c1[8], c2[8];
    o_im_tl(U1, a1);
    o_im_tl(U2, a2);
    o_icomm(a1, a2, c);
    o_icomm(a1, c, c1);
    o_icomm(a2, c, c2);
    for (int a = 0; a < 8; a++) ds[a] = -0.5 * c[a] - 0.375 * c1[a] - 0.125 * c2[a];
}

/* input features of one link pair (unscaled; layout in the header) */
void o_ic_features(const cplx U1[9], const cplx U2[9], double feat[36]) {
    double a1[8], a2[8], c[8], ds[8];
    o_im_tl(U1, a1);
    o_im_tl(U2, a2);
    o_icomm(a1, a2, c);
    o_ic_series(U1, U2, ds);
    double s11 = 0, s22 = 0, s12 = 0, scc = 0;
    for (int a = 0; a < 8; a++) {
        feat[a] = a1[a];
        feat[8 + a] = a2[a];
        feat[16 + a] = c[a];
        feat[24 + a] = ds[a] + 0.5 * c[a];
        s11 += a1[a] * a1[a];
        s22 += a2[a] * a2[a];
        s12 += a1[a] * a2[a];
        scc += c[a] * c[a];
    }
    feat[32] = s11;
    feat[33] = s22;
    feat[34] = s12;
    feat[35] = scc;
}

/* offset of a solution from U1 U2: delta^a = 2 Im Tr[t^a U (U1 U2)^dag] */
void o_ic_delta(const cplx U1[9], const cplx U2[9], const cplx U[9], double delta[8]) {
    cplx P[9], W[9];
    o_mul(U1, U2, P);
    o_mul_dn(U, P, W);
    o_im_tl(W, delta);
}

/* training target of one link (unscaled): delta - delta_s */
void o_ic_target(const cplx U1[9], const cplx U2[9], const cplx U[9], double target[8]) {
    double d[8], ds[8];
    o_ic_delta(U1, U2, U, d);
    o_ic_series(U1, U2, ds);
    for (int a = 0; a < 8; a++) target[a] = d[a] - ds[a];
}

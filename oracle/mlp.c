/*
 * mlp.c -- the oracle's pressure-seed network (10 -> 64 -> 64 -> 1, ReLU).
 *
 * TEST INFRASTRUCTURE ONLY (see mcref.h).
 *
 * The network is not in the paper; it proposes the star pressure that seeds
 * the Newton iteration of the exact Euler solver (exact.c).  Inputs are the
 * ten features of mcref_mlp_features (standardised by the caller and padded
 * with zeros to 16), the output is the log-ratio ln(p*) - ln(p_TR) of the
 * star pressure to the two-rarefaction guess.
 *
 * Precision model of the GPU kernels, reproduced here when bf16 != 0: every
 * GEMM operand (inputs, weights, activations, back-propagated activation
 * gradients) is rounded to bfloat16 (via float, round-to-nearest-even); sums
 * and biases stay wide.  The rounded values are the ones stored in H1, H2.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include "mcref.h"

double mcref_round_bf16(double x)
{
    float f = (float)x;
    uint32_t u;
    memcpy(&u, &f, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return x;  /* inf / nan unchanged */
    u = (u + 0x7fffu + ((u >> 16) & 1u)) & 0xffff0000u;
    memcpy(&f, &u, 4);
    return (double)f;
}

static double rnd(double x, int bf16)
{
    return bf16 ? mcref_round_bf16(x) : x;
}

void mcref_mlp_features(double gamma, double rl, double ul, double pl,
                        double rr, double ur, double pr, double* feat)
{
    double cl = sqrt(gamma * pl / rl), cr = sqrt(gamma * pr / rr);
    double du = ur - ul;
    double ptr = mcref_seed(MCREF_SEED_TR, gamma, rl, ul, pl, rr, ur, pr);
    /* the PV guess without its positivity floor */
    double ppv = 0.5 * (pl + pr) - 0.125 * du * (rl + rr) * (cl + cr);
    const double eps = 1e-6;
    feat[0] = log(rl);
    feat[1] = log(rr);
    feat[2] = log(pl);
    feat[3] = log(pr);
    feat[4] = log(cl);
    feat[5] = log(cr);
    feat[6] = du;
    feat[7] = du / (cl + cr);
    feat[8] = log(ptr);
    feat[9] = log(ppv > eps ? ppv : eps);
}

void mcref_mlp_forward(int64_t B, const double* X, const double* W1, const double* b1,
                       const double* W2, const double* b2, const double* W3, const double* b3,
                       int bf16, double* out, double* H1, double* H2)
{
    const int K = MCREF_KIN, N = MCREF_NH;
    double h1[MCREF_NH], h2[MCREF_NH];
    for (int64_t b = 0; b < B; b++) {
        const double* x = X + b * K;
        for (int j = 0; j < N; j++) {
            double acc = b1[j];
            for (int i = 0; i < K; i++) acc += rnd(x[i], bf16) * rnd(W1[i * N + j], bf16);
            h1[j] = rnd(acc > 0.0 ? acc : 0.0, bf16);
        }
        for (int k = 0; k < N; k++) {
            double acc = b2[k];
            for (int j = 0; j < N; j++) acc += h1[j] * rnd(W2[j * N + k], bf16);
            h2[k] = rnd(acc > 0.0 ? acc : 0.0, bf16);
        }
        double o = b3[0];
        for (int k = 0; k < N; k++) o += h2[k] * rnd(W3[k], bf16);
        out[b] = o;
        if (H1) memcpy(H1 + b * N, h1, sizeof(h1));
        if (H2) memcpy(H2 + b * N, h2, sizeof(h2));
    }
}

double mcref_mlp_backward(int64_t B, const double* X, const double* y,
                          const double* W1, const double* b1, const double* W2, const double* b2,
                          const double* W3, const double* b3, int bf16,
                          double* gW1, double* gb1, double* gW2, double* gb2,
                          double* gW3, double* gb3)
{
    const int K = MCREF_KIN, N = MCREF_NH;
    double* H1 = malloc(sizeof(double) * (size_t)B * N);
    double* H2 = malloc(sizeof(double) * (size_t)B * N);
    double* out = malloc(sizeof(double) * (size_t)B);
    mcref_mlp_forward(B, X, W1, b1, W2, b2, W3, b3, bf16, out, H1, H2);
    memset(gW1, 0, sizeof(double) * K * N);
    memset(gb1, 0, sizeof(double) * N);
    memset(gW2, 0, sizeof(double) * N * N);
    memset(gb2, 0, sizeof(double) * N);
    memset(gW3, 0, sizeof(double) * N);
    gb3[0] = 0.0;
    double loss = 0.0;
    double d2[MCREF_NH], d1[MCREF_NH];
    for (int64_t b = 0; b < B; b++) {
        const double* x = X + b * K;
        const double* h1 = H1 + b * N;
        const double* h2 = H2 + b * N;
        double r = out[b] - y[b];
        loss += r * r;
        double dout = 2.0 * r / (double)B;
        gb3[0] += dout;
        for (int k = 0; k < N; k++) {
            gW3[k] += h2[k] * dout;
            d2[k] = h2[k] > 0.0 ? dout * rnd(W3[k], bf16) : 0.0;
            gb2[k] += d2[k];
        }
        for (int j = 0; j < N; j++) {
            double acc = 0.0;
            for (int k = 0; k < N; k++) {
                double dk = rnd(d2[k], bf16);
                gW2[j * N + k] += h1[j] * dk;
                acc += dk * rnd(W2[j * N + k], bf16);
            }
            d1[j] = h1[j] > 0.0 ? acc : 0.0;
            gb1[j] += d1[j];
        }
        for (int i = 0; i < K; i++)
            for (int j = 0; j < N; j++) gW1[i * N + j] += rnd(x[i], bf16) * rnd(d1[j], bf16);
    }
    free(H1); free(H2); free(out);
    return loss / (double)B;
}

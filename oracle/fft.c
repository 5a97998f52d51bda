/*
 * Mixed-radix complex FFT for the oracle's Poisson solve (test infrastructure).
 *
 * Plain recursive decimation-in-time: X_k = sum_n x_n exp(sign * 2 pi i k n / N),
 * split by the smallest prime factor p of N into p interleaved sub-transforms
 * and recombined with twiddles (Cooley & Tukey 1965, general radix).  Any N
 * works (a prime N degrades to the O(N^2) DFT).  Unnormalised in both
 * directions.  Pinned against numpy.fft.fft2 in tests/test_oracle_ic.py.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle.h"

static int smallest_factor(int n) {
    for (int p = 2; p * p <= n; p++)
        if (n % p == 0) return p;
    return n;
}

static void fft_rec(int n, const cplx *in, int stride, cplx *out, int sign) {
    if (n == 1) { out[0] = in[0]; return; }
    int p = smallest_factor(n);
    int m = n / p;
    cplx *sub = (cplx *)malloc(sizeof(cplx) * n);
    cplx *tw = (cplx *)malloc(sizeof(cplx) * n);
    for (int j = 0; j < n; j++) {
        double ang = sign * 2.0 * M_PI * (double)j / (double)n;
        tw[j] = cos(ang) + I * sin(ang);
    }
    for (int r = 0; r < p; r++) fft_rec(m, in + r * stride, stride * p, sub + r * m, sign);
    for (int q = 0; q < p; q++)
        for (int k = 0; k < m; k++) {
            int kk = k + q * m;
            cplx acc = 0;
            for (int r = 0; r < p; r++) acc += sub[r * m + k] * tw[(long)r * kk % n];
            out[kk] = acc;
        }
    free(tw);
    free(sub);
}

int o_fft2(int n, cplx *a, int sign) {
    cplx *line = (cplx *)malloc(sizeof(cplx) * n);
    cplx *res = (cplx *)malloc(sizeof(cplx) * n);
    if (!line || !res) { free(line); free(res); return -1; }
    /* along x (contiguous) */
    for (int y = 0; y < n; y++) {
        memcpy(line, a + (size_t)n * y, sizeof(cplx) * n);
        fft_rec(n, line, 1, res, sign);
        memcpy(a + (size_t)n * y, res, sizeof(cplx) * n);
    }
    /* along y */
    for (int x = 0; x < n; x++) {
        for (int y = 0; y < n; y++) line[y] = a[x + (size_t)n * y];
        fft_rec(n, line, 1, res, sign);
        for (int y = 0; y < n; y++) a[x + (size_t)n * y] = res[y];
    }
    free(line);
    free(res);
    return 0;
}

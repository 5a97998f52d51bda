/*
 * FP64 reference of the transport coefficients and anisotropy ratios of the
 * momentum broadening (Sec. 2 of arXiv:2307.07999, "Quantifying the effect of
 * Glasma", Eq. 3; test infrastructure, see oracle.h).
 *
 * Input: a broadening table of `rows` rows with `stride` doubles per row, the first
 * four of which are {tau, <dp_x^2>, <dp_y^2>, <dp_z^2>} (tau strictly increasing).
 *
 * Eq. 3 defines the coefficients as the proper-time derivative of the averaged
 * broadening: d<dp_i^2>/dtau.  The paper gives no discretisation; the reading taken
 * is the plain finite-difference derivative on the table's own tau grid:
 *   interior rows:  (f[r+1] - f[r-1]) / (tau[r+1] - tau[r-1])   (central)
 *   first row:      (f[1] - f[0]) / (tau[1] - tau[0])             (forward)
 *   last row:       (f[N-1] - f[N-2]) / (tau[N-1] - tau[N-2])     (backward)
 * A single row has no derivative (0).
 *
 * Heavy quarks (kind 0): the same paragraph fixes the directions with respect to the
 * beam axis, <dp_L^2> = <dp_z^2> and <dp_T^2> = <dp_x^2> + <dp_y^2>, so
 * kappa_T = d<dp_T^2>/dtau, kappa_L = d<dp_z^2>/dtau, and the anisotropy is
 * <dp_L^2> / <dp_T^2>.  Jets along x (kind 1): qhat_y = d<dp_y^2>/dtau,
 * qhat_z = d<dp_z^2>/dtau, anisotropy <dp_z^2> / <dp_y^2>.  The "total" coefficient
 * of the paper's peaks is the sum of the two (reading: kappa_T + kappa_L, and
 * qhat_y + qhat_z).  A ratio whose denominator is zero is NaN.
 *
 * Output rows (8 doubles): {tau, d<dp_x^2>/dtau, d<dp_y^2>/dtau, d<dp_z^2>/dtau,
 * transverse coefficient, longitudinal coefficient, total, anisotropy}.
 *
 * Pins (tests/test_oracle_estimators.py): polynomial tables whose derivatives and
 * ratios are known in closed form (a quadratic is differentiated exactly by the
 * central rule, the end rules give the secant slope), on uniform and uneven grids,
 * for both kinds; variants with a planted mistake (an end rule, a divisor, a swapped
 * direction) are shown to fail the same pins.
 */
#include <math.h>

#include "oracle.h"

void o_derivative(int rows, const double *tau, int tstride, const double *f, int fstride, double *df,
                  int dstride) {
    for (int r = 0; r < rows; r++) {
        int lo = r - 1, hi = r + 1;
        if (lo < 0) lo = 0;
        if (hi > rows - 1) hi = rows - 1;
        if (hi == lo) {
            df[(long)r * dstride] = 0.0;
            continue;
        }
        df[(long)r * dstride] = (f[(long)hi * fstride] - f[(long)lo * fstride]) /
                                (tau[(long)hi * tstride] - tau[(long)lo * tstride]);
    }
}

void o_transport_coefficients(int rows, const double *tab, int stride, int kind, double *out) {
    for (int r = 0; r < rows; r++) out[8 * r] = tab[(long)r * stride];
    for (int i = 0; i < 3; i++) o_derivative(rows, tab, stride, tab + 1 + i, stride, out + 1 + i, 8);
    for (int r = 0; r < rows; r++) {
        double *o = out + 8 * r;
        const double *t = tab + (long)r * stride;
        double trans, lon, den;
        if (kind == 0) {
            trans = o[1] + o[2];
            lon = o[3];
            den = t[1] + t[2];
        } else {
            trans = o[2];
            lon = o[3];
            den = t[2];
        }
        o[4] = trans;
        o[5] = lon;
        o[6] = trans + lon;
        o[7] = den != 0.0 ? t[3] / den : NAN;
    }
}

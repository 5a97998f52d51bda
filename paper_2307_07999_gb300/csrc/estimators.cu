// Transport coefficients and anisotropy ratios of the momentum broadening (Sec. 2 of
// arXiv:2307.07999, "Quantifying the effect of Glasma", Eq. 3): kappa_i (heavy quarks,
// i in {L, T}) and qhat_i (jets along x, i in {z, y}) are the proper-time derivatives
// of the event- and particle-averaged <dp_i^2>(tau).  The GPU produces the FP64 sums of
// <dp_i^2> per step (broadening tables); this is the derivative of such a table, a few
// hundred rows, so it runs on the host in FP64 inside the library.
#include <math.h>
#include <stdint.h>

#include "../../include/glasma.h"

void glasma_set_error(const char* msg);

namespace {

// slope of column col between rows a < b
inline double slope(const double* t, int64_t stride, int col, int64_t a, int64_t b) {
    return (t[b * stride + col] - t[a * stride + col]) / (t[b * stride] - t[a * stride]);
}

}  // namespace

extern "C" glasma_status broadening_transport(const double* table, int64_t rows, int32_t stride, int32_t kind,
                                              double* out) {
    if (!table || !out || rows < 1 || stride < 4 || (kind != GLASMA_HEAVY_QUARKS && kind != GLASMA_JETS_X)) {
        glasma_set_error("broadening_transport: bad arguments");
        return GLASMA_ERR_INVALID;
    }
    for (int64_t r = 1; r < rows; r++)
        if (!(table[r * stride] > table[(r - 1) * stride])) {
            glasma_set_error("broadening_transport: tau must increase strictly");
            return GLASMA_ERR_INVALID;
        }
    for (int64_t r = 0; r < rows; r++) {
        const double* row = table + r * stride;
        double* o = out + 8 * r;
        o[0] = row[0];
        // centred stencil inside the table, the one-sided secant at its two ends
        const int64_t a = r > 0 ? r - 1 : 0, b = r + 1 < rows ? r + 1 : rows - 1;
        for (int c = 1; c <= 3; c++) o[c] = a == b ? 0.0 : slope(table, stride, c, a, b);
        // heavy quarks: T = x + y, L = z (beam axis); jets along x: transverse y, longitudinal z
        const double tr = kind == GLASMA_HEAVY_QUARKS ? o[1] + o[2] : o[2];
        const double den = kind == GLASMA_HEAVY_QUARKS ? row[1] + row[2] : row[2];
        o[4] = tr;
        o[5] = o[3];
        o[6] = tr + o[3];
        o[7] = den == 0.0 ? NAN : row[3] / den;
    }
    return GLASMA_OK;
}

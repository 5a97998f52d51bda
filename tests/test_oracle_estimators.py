"""Pins of the oracle's Eq. 3 estimators (oracle/estimators.c).

Eq. 3 of the paper (Sec. 2, "Quantifying the effect of Glasma") defines kappa_i and
qhat_i as d<dp_i^2>/dtau, with L = z and T = x + y for heavy quarks and the z, y
directions for jets along x, and the anisotropy as the longitudinal over the transverse
broadening.  The tables below are polynomials in tau, for which the finite-difference
derivative of the oracle's reading (central inside, one-sided at the ends) is known in
closed form: the central rule differentiates a quadratic exactly at the midpoint of its
stencil only on a uniform grid, and on any grid it returns the secant slope
b + c (tau_lo + tau_hi) of f = a + b tau + c tau^2.  The same pins are applied to
variants of the estimator with a planted mistake, each of which must fail one of them.
"""
import math

import numpy as np
import pytest

import oracle as O


def _table(tau, coef):
    """rows {tau, f_x, f_y, f_z, count} with f_i = a_i + b_i tau + c_i tau^2"""
    t = np.zeros((len(tau), 5))
    t[:, 0] = tau
    for i, (a, b, c) in enumerate(coef):
        t[:, 1 + i] = a + b * tau + c * tau ** 2
    t[:, 4] = 1000.0
    return t


def _secant(tau, coef):
    """closed-form secant slopes on each row's stencil: d_i[r] = b_i + c_i (tau_lo + tau_hi)"""
    n = len(tau)
    lo = np.maximum(np.arange(n) - 1, 0)
    hi = np.minimum(np.arange(n) + 1, n - 1)
    d = np.zeros((n, 3))
    for i, (a, b, c) in enumerate(coef):
        d[:, i] = b + c * (tau[lo] + tau[hi])
    return d


COEF = [(0.0, 0.7, 1.9), (0.0, 1.3, -0.4), (0.0, 2.9, 0.35)]  # distinct per direction
GRIDS = {
    "uniform": 0.0125 * np.arange(3, 40),
    "uneven": np.cumsum(np.r_[0.05, 0.01 + 0.02 * np.abs(np.sin(np.arange(1, 31)))]),
}


def pin_failures(est):
    """Runs every pin on est(table, kind) -> rows {tau, dx, dy, dz, transverse,
    longitudinal, total, anisotropy}; returns the names of the pins that fail."""
    bad = []
    for gname, tau in GRIDS.items():
        tab = _table(tau, COEF)
        want_d = _secant(tau, COEF)
        for kind in ("hq", "jet"):
            out = np.asarray(est(tab, kind))
            if not np.allclose(out[:, 0], tau, rtol=0, atol=0):
                bad.append(f"{gname}/{kind}: tau column")
            if not np.allclose(out[:, 1:4], want_d, rtol=1e-12, atol=1e-12):
                bad.append(f"{gname}/{kind}: derivative")
            if kind == "hq":
                tr, lon = want_d[:, 0] + want_d[:, 1], want_d[:, 2]
                ratio = tab[:, 3] / (tab[:, 1] + tab[:, 2])
            else:
                tr, lon = want_d[:, 1], want_d[:, 2]
                ratio = tab[:, 3] / tab[:, 2]
            if not np.allclose(out[:, 4], tr, rtol=1e-12, atol=1e-12):
                bad.append(f"{gname}/{kind}: transverse")
            if not np.allclose(out[:, 5], lon, rtol=1e-12, atol=1e-12):
                bad.append(f"{gname}/{kind}: longitudinal")
            if not np.allclose(out[:, 6], tr + lon, rtol=1e-12, atol=1e-12):
                bad.append(f"{gname}/{kind}: total")
            if not np.allclose(out[:, 7], ratio, rtol=1e-12, atol=0, equal_nan=True):
                bad.append(f"{gname}/{kind}: anisotropy")
    # a uniform grid differentiates a quadratic exactly at interior rows
    tau = GRIDS["uniform"]
    out = np.asarray(est(_table(tau, COEF), "hq"))
    for i, (a, b, c) in enumerate(COEF):
        if not np.allclose(out[1:-1, 1 + i], b + 2 * c * tau[1:-1], rtol=1e-12, atol=1e-12):
            bad.append("uniform interior exact")
    # a linear table has its slope everywhere, end rows included
    lin = _table(tau, [(0.3, 1.1, 0.0), (0.0, -0.2, 0.0), (1.0, 4.0, 0.0)])
    out = np.asarray(est(lin, "hq"))
    if not np.allclose(out[:, 1:4], np.tile([1.1, -0.2, 4.0], (len(tau), 1)), rtol=1e-12, atol=1e-12):
        bad.append("linear slope")
    # zero transverse broadening (the formation row): the ratio is undefined
    z = _table(tau[:4], COEF)
    z[0, 1:4] = 0.0
    out = np.asarray(est(z, "hq"))
    if not math.isnan(out[0, 7]):
        bad.append("NaN at zero denominator")
    return bad


def test_oracle_estimators_meet_their_pins():
    assert pin_failures(O.transport_coefficients) == []


def test_single_row_has_zero_derivative():
    out = O.transport_coefficients(np.array([[0.1, 0.5, 0.5, 0.2, 10.0]]))
    assert np.all(out[0, 1:7] == 0.0)


def test_kappa_scales_with_units():
    # kappa in GeV^2/fm: a table in GeV^2 against tau in fm scaled by s in tau divides kappa by s
    tau = GRIDS["uniform"]
    tab = _table(tau, COEF)
    k1 = O.kappa_qhat(tab)
    tab2 = tab.copy()
    tab2[:, 0] *= 2.5
    k2 = O.kappa_qhat(tab2)
    assert np.allclose(k2[:, 1:], k1[:, 1:] / 2.5, rtol=1e-13)


# ------------------------------------------------------------------ planted mistakes
def _ref(tab, kind):
    return O.transport_coefficients(tab, kind)


def _mut_central_ends(tab, kind):
    # end rows taken as a central difference with the grid wrapped around
    out = _ref(tab, kind).copy()
    t, f = tab[:, 0], tab[:, 1:4]
    out[0, 1:4] = (f[1] - f[-1]) / (t[1] - t[-1])
    return _recombine(out, tab, kind)


def _mut_zero_ends(tab, kind):
    out = _ref(tab, kind).copy()
    out[0, 1:4] = 0.0
    out[-1, 1:4] = 0.0
    return _recombine(out, tab, kind)


def _mut_half_step(tab, kind):
    # interior divided by one grid step instead of the stencil width
    out = _ref(tab, kind).copy()
    t, f = tab[:, 0], tab[:, 1:4]
    out[1:-1, 1:4] = (f[2:] - f[:-2]) / (t[1:-1, None] - t[:-2, None])
    return _recombine(out, tab, kind)


def _mut_forward_everywhere(tab, kind):
    out = _ref(tab, kind).copy()
    t, f = tab[:, 0], tab[:, 1:4]
    out[:-1, 1:4] = (f[1:] - f[:-1]) / (t[1:, None] - t[:-1, None])
    return _recombine(out, tab, kind)


def _mut_transverse_x_only(tab, kind):
    out = _ref(tab, kind).copy()
    if kind == "hq":
        out[:, 4] = out[:, 1]
        out[:, 6] = out[:, 4] + out[:, 5]
    return out


def _mut_jet_uses_x(tab, kind):
    out = _ref(tab, kind).copy()
    if kind == "jet":
        out[:, 4] = out[:, 1]
        out[:, 6] = out[:, 4] + out[:, 5]
        out[:, 7] = tab[:, 3] / tab[:, 1]
    return out


def _mut_inverted_ratio(tab, kind):
    out = _ref(tab, kind).copy()
    out[:, 7] = 1.0 / out[:, 7]
    return out


def _recombine(out, tab, kind):
    if kind == "hq":
        out[:, 4] = out[:, 1] + out[:, 2]
    else:
        out[:, 4] = out[:, 2]
    out[:, 5] = out[:, 3]
    out[:, 6] = out[:, 4] + out[:, 5]
    return out


@pytest.mark.parametrize("mutant", [_mut_central_ends, _mut_zero_ends, _mut_half_step, _mut_forward_everywhere,
                                    _mut_transverse_x_only, _mut_jet_uses_x, _mut_inverted_ratio])
def test_planted_mistakes_fail_the_pins(mutant):
    assert pin_failures(mutant), f"{mutant.__name__} passed every pin"

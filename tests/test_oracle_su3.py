"""Pins of the oracle's SU(3) algebra against closed forms, tables and libraries.

The color algebra is the one of Sec. 1 ("Probes in Glasma"): Q = Q^a T^a,
q2 = Q^a Q^a, q3 = d_abc Q^a Q^b Q^c with the SU(3) generators T^a.
"""
import itertools
import os

import numpy as np
import pytest
import scipy.linalg as sl

import oracle as O
from conftest import GOLDEN


def _load_structure():
    f = np.zeros((8, 8, 8))
    d = np.zeros((8, 8, 8))
    for line in open(os.path.join(GOLDEN, "su3_structure_constants.txt")):
        if line.startswith("#") or not line.strip():
            continue
        k, a, b, c, v = line.split()
        a, b, c, v = int(a) - 1, int(b) - 1, int(c) - 1, float(v)
        for p in set(itertools.permutations((a, b, c))):
            if k == "f":
                sign = np.linalg.det(np.eye(3)[[list((a, b, c)).index(q) for q in p]])
                f[p] = v * sign
            else:
                d[p] = v
    return f, d


def test_generators_orthonormal_hermitian_traceless():
    T = [O.generator(a) for a in range(8)]
    for a in range(8):
        assert np.allclose(T[a], T[a].conj().T, atol=1e-15)
        assert abs(np.trace(T[a])) < 1e-15
        for b in range(8):
            assert abs(np.trace(T[a] @ T[b]) - 0.5 * (a == b)) < 1e-15


def test_structure_constants_match_table():
    f_ref, d_ref = _load_structure()
    f, d = O.structure_constants()
    assert np.abs(f - f_ref).max() < 1e-14
    assert np.abs(d - d_ref).max() < 1e-14
    # sum rules: f_abc f_abd = 3 delta_cd (C_A = N), d_abc d_abc = (N^2-4)(N^2-1)/N = 40/3
    assert np.allclose(np.einsum("abc,abd->cd", f, f), 3 * np.eye(8), atol=1e-13)
    assert abs((d ** 2).sum() - 40.0 / 3.0) < 1e-12


def test_algebra_roundtrip_and_imtl():
    rng = np.random.default_rng(0)
    x = rng.standard_normal(8)
    X = O.alg_to_mat(x)
    assert np.allclose(O.mat_to_alg(X), x, atol=1e-15)
    # ImTL of exp(i e X) = e X + O(e^3)
    e = 1e-4
    P = sl.expm(1j * e * X)
    assert np.allclose(O.im_tl(P) / e, x, atol=1e-7)
    # ImTL of a general matrix: components of [(P - P^dag)/(2i)] traceless part
    M = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))
    H = (M - M.conj().T) / 2j
    H -= np.trace(H) / 3 * np.eye(3)
    assert np.allclose(O.alg_to_mat(O.im_tl(M)), H, atol=1e-14)


def test_exp_against_scipy_and_abelian_closed_form():
    rng = np.random.default_rng(1)
    for scale in (1e-3, 0.3, 2.0, 7.0):
        x = scale * rng.standard_normal(8)
        U = O.exp_i(x)
        R = sl.expm(1j * O.alg_to_mat(x))
        assert np.abs(U - R).max() < 5e-14 * max(1.0, scale)
        assert O.unitarity_dev(U) < 1e-13
    th = 0.9
    x = np.zeros(8)
    x[2] = th
    assert np.allclose(O.exp_i(x), np.diag([np.exp(0.5j * th), np.exp(-0.5j * th), 1.0]), atol=1e-15)


def test_transport_is_conjugation():
    rng = np.random.default_rng(2)
    U = O.exp_i(rng.standard_normal(8))
    x = rng.standard_normal(8)
    X = O.alg_to_mat(x)
    assert np.allclose(O.alg_to_mat(O.transport(U, x)), U.conj().T @ X @ U, atol=1e-14)
    assert np.allclose(O.alg_to_mat(O.conj_by(U, x)), U @ X @ U.conj().T, atol=1e-14)


def test_haar_moments():
    # Mezzadri (2007): E|U_ij|^2 = 1/3, E U_ij = 0, E |U_ij|^4 = 1/6 for U(3) Haar
    rng = np.random.default_rng(3)
    m = 20000
    us = np.array([O.haar(rng.standard_normal(18)) for _ in range(m)])
    assert np.abs(us.mean(0)).max() < 5 * np.sqrt(1 / 3 / m)
    a2 = (np.abs(us) ** 2).mean(0)
    assert np.abs(a2 - 1 / 3).max() < 5 * np.sqrt((1 / 6 - 1 / 9) / m)
    for u in us[:50]:
        assert np.allclose(u @ u.conj().T, np.eye(3), atol=1e-14)


def test_reunitarize():
    rng = np.random.default_rng(4)
    U = O.exp_i(rng.standard_normal(8))
    Up = U + 1e-6 * (rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3)))
    R = O.reunitarize(Up)
    assert O.unitarity_dev(R) < 1e-15 * 10
    assert np.abs(R - U).max() < 1e-5
    # an exact SU(3) element is a fixed point
    assert np.abs(O.reunitarize(U) - U).max() < 1e-14


def test_cartan_charge_casimirs():
    # Sec. 1: <Q^a Q^b> = delta/2, <Q^a Q^b Q^c> = d^abc / 4  =>  q2 = 4, q3 = 10/3
    Q0 = O.q0_cartan(4.0, 10.0 / 3.0)
    q2, q3 = O.casimirs(Q0)
    assert abs(q2 - 4.0) < 1e-14 and abs(q3 - 10.0 / 3.0) < 1e-13
    assert np.count_nonzero(Q0[[0, 1, 3, 4, 5, 6]]) == 0
    # matrix forms q2 = 2 Tr Q^2 and q3 = 4 Tr Q^3
    Qm = O.alg_to_mat(Q0)
    assert abs(2 * np.trace(Qm @ Qm).real - 4.0) < 1e-13
    assert abs(4 * np.trace(Qm @ Qm @ Qm).real - 10.0 / 3.0) < 1e-13

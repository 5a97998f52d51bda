"""Shared helpers for the GPU parity tests: seeded synthetic inputs and the
comparison metric.  No physics here; both the oracle and the CUDA path consume
the same inputs."""
import numpy as np

import oracle as O

HBARC = 0.1973269804


def rel_err(got, want):
    """max |got - want| / max |want| (normwise; element-wise relative errors are
    ill-conditioned for components near zero)."""
    got = np.asarray(got)
    want = np.asarray(want)
    den = np.abs(want).max()
    return np.abs(got - want).max() / (den if den > 0 else 1.0)


def random_state(n, seed, step=3, link_scale=0.7, e_scale=0.4, phi_scale=0.3):
    """Random links exp(i x.t), random E, phi, pi (seeded)."""
    rng = np.random.default_rng(seed)
    st = O.State(n, step=step)
    for s in range(n * n):
        for d in range(2):
            st.U[s, d] = O.exp_i(link_scale * rng.standard_normal(8))
    st.E[...] = e_scale * rng.standard_normal((n * n, 2, 8))
    st.phi[...] = phi_scale * rng.standard_normal((n * n, 8))
    st.pi[...] = e_scale * rng.standard_normal((n * n, 8))
    return st


def random_particles(np_, n, seed, pscale=0.6, mass=0.5, peta=True):
    rng = np.random.default_rng(seed)
    P = O.Particles(np_)
    P.x[:] = rng.uniform(0, n, np_)
    P.y[:] = rng.uniform(0, n, np_)
    P.px[:] = pscale * rng.standard_normal(np_)
    P.py[:] = pscale * rng.standard_normal(np_)
    if peta:
        P.peta[:] = 0.3 * pscale * rng.standard_normal(np_)
    Q0 = O.q0_cartan()
    for j in range(np_):
        P.Q[j] = O.conj_by(O.haar(rng.standard_normal(18)), Q0)
    P.set_p0(mass)
    return P


def lattice_units(n, L_fm, g2mu=2.0, mir=0.2):
    a_fm = L_fm / n
    a = a_fm / HBARC
    return a_fm, a, g2mu * a, mir * a

"""Seeded synthetic workloads (input recipes only; no arithmetic of the method).

The paper's workloads are synthetic by construction: MV-model random color
charges with a fixed g^2 mu, and toy-model particle ensembles (Sec. 2,
"Quantifying the effect of Glasma").  Seeds: Philox key of event e of
workload w is w * 2^32 + e (+ 1000 * rank for independent replicas); the
particle key is that key xor 0x5A5A5A5A5A5A5A5A.
"""
import numpy as np

from ._lib import GLASMA_FP32, GLASMA_FP64, CpicParams, GlasmaParams

HBARC = 0.1973269804  # GeV fm
PARTICLE_KEY_XOR = 0x5A5A5A5A5A5A5A5A


def event_seed(workload, event, rank=0):
    return (workload << 32) + event + 1000 * rank


def glasma_params(n, L_fm, g2mu, seed, precision, tau_end_fm=1.0, m_ir=0.2, n_sheets=10, reunit_every=64):
    return GlasmaParams(n, n_sheets, L_fm, g2mu, m_ir, 0.125, tau_end_fm, precision, reunit_every, 1, 100, 1e-12,
                        seed)


def charm_params(n_particles, seed, mass=1.5, p_max=5.0, tau_form=None, integrator=0):
    # tau_form = 1/(2M) (Sec. 2: formation time proportional to the inverse mass)
    tf = HBARC / (2.0 * mass) if tau_form is None else tau_form
    return CpicParams(n_particles, 0, mass, tf, 0.0, p_max, 4.0, 10.0 / 3.0, 0, integrator, 1, 0, seed ^ PARTICLE_KEY_XOR)


def batched_uneven(rank=0, precision=GLASMA_FP32, n_events=64, sizes=(128, 256, 384, 512), n_particles=10000):
    """64 events of uneven lattices (16 each of 128^2, 256^2, 384^2, 512^2), L = 10 fm,
    g^2 mu ~ U[1.5, 2.5] GeV per event, m_IR = 0.2 GeV, 10 sheets, dtau = a/8 to
    tau = 1 fm/c; 10k charm quarks per event (M = 1.5 GeV, |p_T| ~ U[0, 5] GeV,
    isotropic azimuth, tau_form = 1/(2M))."""
    rng = np.random.default_rng(event_seed(3, 0, rank))
    g2mu = 1.5 + rng.random(n_events)
    per = n_events // len(sizes)
    evs, pps = [], []
    for e in range(n_events):
        n = sizes[min(e // per, len(sizes) - 1)]
        s = event_seed(3, e, rank)
        evs.append(glasma_params(n, 10.0, float(g2mu[e]), s, precision))
        pps.append(charm_params(n_particles, s))
    return evs, pps


def single_32(precision=GLASMA_FP64):
    """32^2, L = 6 fm, g^2 mu = 2 GeV, 1000 charm at rest formed at 0.1 fm/c."""
    s = event_seed(1, 0)
    return ([glasma_params(32, 6.0, 2.0, s, precision, reunit_every=0)],
            [CpicParams(1000, 0, 1.5, 0.1, 0.0, 0.0, 4.0, 10.0 / 3.0, 0, 0, 1, 0, s ^ PARTICLE_KEY_XOR)])


WORKLOADS = {"batched_uneven": batched_uneven, "single_32": single_32}
__all__ = ["batched_uneven", "single_32", "glasma_params", "charm_params", "event_seed", "GLASMA_FP32", "GLASMA_FP64"]

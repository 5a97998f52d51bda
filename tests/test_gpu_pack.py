"""Several ensembles on one event: cpic_push_many pushes the ensembles on the default kernel
(one particle step per field step, nearest-grid-point gather) in shared launches, their
blocks interleaved, up to eight per launch; the others alone.  Every ensemble must come out
exactly as when it is pushed alone on an identical copy of the event: the same particles
bit for bit (the per-particle arithmetic is the same) and the same broadening table up to
the order of the FP64 block sums."""
import numpy as np
import pytest

from gpu_common import rel_err

pytestmark = pytest.mark.gpu

G = pytest.importorskip("paper_2307_07999_gb300")

# (n_particles, mass GeV, tau_form fm, p range GeV, init_kind, integrator, substeps, bin_every, interp)
SPECS = [
    (300, 1.5, 0.05, (0.0, 3.0), 0, 0, 1, 0, 0),
    (128, 4.7, 0.02, (0.0, 5.0), 0, 1, 1, 0, 0),    # Boris kick, exactly one block
    (257, 0.0, 0.0, (5.0, 5.0), 1, 0, 1, 2, 0),     # massless along x, sorted every 2 steps
    (1, 1.5, 0.08, (0.0, 2.0), 0, 0, 1, 0, 0),      # a single particle
    (0, 1.5, 0.05, (0.0, 3.0), 0, 0, 1, 0, 0),      # empty
    (700, 1.5, 0.03, (0.0, 3.0), 0, 0, 1, 3, 0),
    (90, 4.7, 0.05, (1.0, 4.0), 0, 1, 1, 0, 0),
    (400, 0.0, 0.0, (2.0, 2.0), 1, 0, 1, 0, 0),
    (333, 1.5, 0.05, (0.0, 3.0), 0, 0, 1, 1, 0),
    (64, 4.7, 0.0, (0.0, 1.0), 0, 1, 1, 0, 0),      # the ninth non-empty one on the default kernel: a second launch
    (150, 1.5, 0.05, (0.0, 3.0), 0, 0, 2, 0, 0),    # sub-stepped: pushed alone
    (150, 1.5, 0.05, (0.0, 3.0), 0, 0, 1, 0, 1),    # cloud in cell: pushed alone
]


def event(prec):
    g = G.Glasma(24, 2.4, g2mu_GeV=1.8, precision=prec, tau_end_fm=0.25, seed=11,
                 reunit_every=(0 if prec == 0 else 16))
    g.init()
    return g


def ensemble(g, k, spec):
    np_, m, tf, (p0, p1), kind, integ, sub, be, interp = spec
    c = G.CPIC(g, np_, m, tf, p_min_GeV=p0, p_max_GeV=p1, init_kind=kind, integrator=integ, substeps=sub,
               bin_every=be, interp=interp, seed=1000 + 17 * k)
    c.init()
    return c


@pytest.mark.parametrize("prec", [0, 1])
def test_ensembles_pushed_together_match_pushed_alone(prec):
    steps = 18
    g = event(prec)
    cs = [ensemble(g, k, s) for k, s in enumerate(SPECS)]
    G.push_many(cs, steps)
    for k, spec in enumerate(SPECS):
        g1 = event(prec)
        c1 = ensemble(g1, k, spec)
        G.push_many([c1], steps)
        a, b = cs[k].broadening(), c1.broadening()
        assert a.shape == b.shape
        assert np.all(a[:, 4] == b[:, 4])
        if spec[0] > 0:
            assert rel_err(a[:, 1:4], b[:, 1:4]) < 1e-13, k
        pa, pb = cs[k].get_particles(), c1.get_particles()
        for key in pa:
            assert np.array_equal(pa[key], pb[key]), (k, key)

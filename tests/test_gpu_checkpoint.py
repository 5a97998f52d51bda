"""Checkpoint and resume of a coupled run through the C ABI: a run stopped at some
step, written to host blobs and continued in freshly created contexts repeats the
uninterrupted run bit for bit (particles, fields), and its broadening tables to the
order of the FP64 atomic sums."""
import numpy as np
import pytest

from gpu_common import rel_err

pytestmark = pytest.mark.gpu

G = pytest.importorskip("paper_2307_07999_gb300")

N, L = 48, 4.0


def event(prec):
    g = G.Glasma(N, L, precision=prec, tau_end_fm=1.0, seed=77, reunit_every=(16 if prec else 0))
    return g


def ensembles(g):
    # two species in one event: explicit kick with sorting every 3 steps, Boris kick
    a = G.CPIC(g, 700, 1.5, 0.03, p_max_GeV=3.0, bin_every=3, seed=5)
    b = G.CPIC(g, 333, 4.7, 0.01, p_max_GeV=3.0, seed=6, integrator=1)
    return [a, b]


@pytest.mark.parametrize("prec", [0, 1])
def test_resume_repeats_the_run(prec):
    g = event(prec)
    assert g.init()[0] == 0
    cs = ensembles(g)
    for c in cs:
        c.init()
    G.push_many(cs, 20)
    blob_g = g.export_state()
    blobs = [c.export_state() for c in cs]
    G.push_many(cs, 31)
    want = [(c.get_particles(), c.broadening()) for c in cs]
    want_U = g.get_state()

    # fresh contexts with the same parameters, resumed from the blobs
    g2 = event(prec)
    cs2 = ensembles(g2)
    g2.import_state(blob_g)
    for c, b in zip(cs2, blobs):
        c.import_state(b)
    G.push_many(cs2, 31)
    for c, (wp, wt) in zip(cs2, want):
        got = c.get_particles()
        for k in wp:
            assert np.array_equal(got[k], wp[k]), k
        t = c.broadening()
        assert t.shape == wt.shape and np.array_equal(t[:, 0], wt[:, 0]) and np.array_equal(t[:, 4], wt[:, 4])
        assert rel_err(t[:, 1:4], wt[:, 1:4]) < 1e-13
    U2 = g2.get_state()
    assert U2[4] == want_U[4]
    for a, b in zip(U2[:4], want_U[:4]):
        assert np.array_equal(a, b)


def test_import_rejects_other_shapes():
    g = event(0)
    assert g.init()[0] == 0
    cs = ensembles(g)
    for c in cs:
        c.init()
    blob_g = g.export_state()
    blob_c = cs[0].export_state()
    other = G.Glasma(N + 2, L, precision=0, tau_end_fm=1.0)
    with pytest.raises(G.GlasmaError):
        other.import_state(blob_g)
    with pytest.raises(G.GlasmaError):
        event(1).import_state(blob_g)   # other precision
    with pytest.raises(G.GlasmaError):
        cs[1].import_state(blob_c)      # other particle count and mass
    bad = blob_g.copy()
    bad[:8] = 0                         # not a checkpoint
    with pytest.raises(G.GlasmaError):
        g.import_state(bad)
    with pytest.raises(G.GlasmaError):
        g.import_state(blob_g[:100])    # truncated
    # a rejected import changes nothing
    s0 = g.get_state()
    g.step(2)
    g.import_state(blob_g)
    s1 = g.get_state()
    assert s1[4] == s0[4] and np.array_equal(s1[0], s0[0])

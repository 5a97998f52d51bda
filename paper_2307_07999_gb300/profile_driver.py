"""Small fixed workloads for ncu captures (one short run each, a few GB at most).

  python -m paper_2307_07999_gb300.profile_driver field 512          # 4 FP32 field steps on 512^2
  python -m paper_2307_07999_gb300.profile_driver push 512 100000    # + a 100k-particle push
  python -m paper_2307_07999_gb300.profile_driver jets 1024 1000000 16   # 40 coupled steps of 1M
    massless partons (|p_x| = 5 GeV, formed at tau = 0) sorted by cell every 16 steps
  python -m paper_2307_07999_gb300.profile_driver batch              # one graph run of the 64-event batch
  python -m paper_2307_07999_gb300.profile_driver batch8             # 8 events of 384^2, 10k charm each
    (both batch workloads tune the field tile shape first: 8 variants x 5 field launches;
     an argument v=<k> sets field tile variant k instead, without tuning, and p=<k> the
     batched push kernel k, e.g. p=2 for the record push; m=<mode> runs the batch in that
     mode (graph, eager, per_event, persistent) and n=<count> gives every event that many
     particles)
  python -m paper_2307_07999_gb300.profile_driver ic 1024            # tau = 0+ solve: cold, then warm start
  python -m paper_2307_07999_gb300.profile_driver corr 512           # 4 FP32 field steps with both correlators
"""
import sys

import torch

from . import Batch, CPIC, Glasma
from . import workloads as W


def main(argv):
    what = argv[1] if len(argv) > 1 else "field"
    if what in ("batch", "batch8"):
        opt = {a.split("=")[0]: a.split("=")[1] for a in argv[2:] if "=" in a}
        npart = int(opt.get("n", 10000))
        evs, pps = (W.batched_uneven(n_particles=npart) if what == "batch"
                    else W.batched_uneven(n_events=8, sizes=(384,), n_particles=npart))
        B = Batch(evs, pps)
        B.init()
        fixed = [a for a in argv[2:] if a.startswith("v=")]
        if fixed:
            B.set_variant(int(fixed[0][2:]))
        else:
            B.tune(steps=4)  # the tile shape bench.py would run (8 variants x 5 launches first)
        push = [a for a in argv[2:] if a.startswith("p=")]
        if push:
            B.set_push_variant(int(push[0][2:]))
        B.run(opt.get("m", "graph"))
        torch.cuda.synchronize()
        print("ok")
        return
    n = int(argv[2]) if len(argv) > 2 else 512
    if what == "ic":
        from . import WarmStartNet, ic_dataset, init_warm
        g = Glasma(n, 10.0, precision=1, tau_end_fm=1.0, seed=3)
        g.init()
        net = WarmStartNet(seed=1)
        X, T = ic_dataset(g)  # a quick fit on this event's own links (profiling only)
        net.fit_scales(X, T)
        net.train(X, T, epochs=2, batch=16384, lr=2e-3)
        init_warm(Glasma(n, 10.0, precision=1, tau_end_fm=1.0, seed=3), net)
        torch.cuda.synchronize()
        print("ok")
        return
    if what == "jets":
        g = Glasma(n, 10.0, precision=1, tau_end_fm=1.0, seed=3, reunit_every=64)
        g.init()
        c = CPIC(g, int(argv[3]) if len(argv) > 3 else 1000000, 0.0, 0.0, p_min_GeV=5.0, p_max_GeV=5.0,
                 init_kind=1, bin_every=int(argv[4]) if len(argv) > 4 else 16, seed=4)
        c.init()
        c.push(40)
        torch.cuda.synchronize()
        print("ok")
        return
    g = Glasma(n, 10.0, precision=1, tau_end_fm=1.0, seed=3)
    g.init()
    if what == "corr":
        from . import Correlators
        c = Correlators(g, tau_start_fm=0.0, ox0=0.5)
        g.step(4)
        torch.cuda.synchronize()
        print("ok")
        return
    g.step(4)
    if what == "push":
        c = CPIC(g, int(argv[3]) if len(argv) > 3 else 100000, 1.5, 0.0, p_max_GeV=5.0, bin_every=1, seed=4)
        c.init()
        c.push(3)
    torch.cuda.synchronize()
    print("ok")


if __name__ == "__main__":
    main(sys.argv)

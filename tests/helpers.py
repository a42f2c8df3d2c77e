"""Shared test helpers (no method arithmetic)."""
import numpy as np

import oracle


def make_oracle(wl, **over):
    w = dict(wl)
    w.update(over)
    strat = {"sp1": oracle.SP1, "sp2": oracle.SP2, "wp": oracle.WP}[w["strategy"]]
    return oracle.Oracle(hbar=w["hbar"], mass=w["mass"], dt=w["dt"],
                         gamma0=w["gamma0"], H=w["H"], w=w["w"], xc=w["xc"],
                         nx=w["nx"], nk=w["nk"], xmin=w["xmin"],
                         xmax=w["xmax"], kmin=w["kmin"], kmax=w["kmax"],
                         strategy=strat, n_alpha=w["n_alpha"], seed=w["seed"],
                         instance=w.get("instance", 0),
                         tangent=w.get("tangent", False),
                         tquantum=w.get("tquantum", 1.0),
                         comps=tuple(w.get("comps", ())),
                         threads=w.get("threads", 1))


def net_sign(w):
    return int(np.sum(np.sign(w)))


def make_oracle4(wl, **over):
    """The 4D Helium-like oracle for a workload dict (workloads.HE_4D_*)."""
    w = dict(wl)
    w.update(over)
    return oracle.Oracle4(hbar=w["hbar"], mass=w["mass"], dt=w["dt"], Z=w["Z"], a=w["a"],
                          xc=w["xc"], lam=w["lam"], nx=w["nx"], nk=w["nk"], xmin=w["xmin"],
                          xmax=w["xmax"], kmin=w["kmin"], kmax=w["kmax"], ny=w["ny"],
                          nkap=w["nkap"], n_alpha=w["n_alpha"], seed=w["seed"])

"""Shared test helpers (no method arithmetic)."""
import numpy as np

import oracle


def make_oracle(wl, **over):
    w = dict(wl)
    w.update(over)
    strat = {"sp1": oracle.SP1, "sp2": oracle.SP2}[w["strategy"]]
    return oracle.Oracle(hbar=w["hbar"], mass=w["mass"], dt=w["dt"],
                         gamma0=w["gamma0"], H=w["H"], w=w["w"], xc=w["xc"],
                         nx=w["nx"], nk=w["nk"], xmin=w["xmin"],
                         xmax=w["xmax"], kmin=w["kmin"], kmax=w["kmax"],
                         strategy=strat, n_alpha=w["n_alpha"], seed=w["seed"],
                         instance=w.get("instance", 0))


def net_sign(w):
    return int(np.sum(np.sign(w)))

"""Helpers of the GPU parity tests: one PDHG evaluation of the CUDA library and of the
oracle from the same iterate state, compared element by element per cone role."""
import numpy as np


def role_masks(prob):
    """Row masks of the cone roles: scalar rows (zero, nonnegative), SOC / RSOC rows, exp rows."""
    m = int(prob["m"])
    kinds = np.repeat(np.asarray(prob["cone_types"]), np.asarray(prob["cone_dims"]))
    assert kinds.size == m
    return {"scalar": kinds <= 1, "soc": (kinds == 2) | (kinds == 3), "exp": kinds >= 4}


def _rel(a, b, mask=None):
    if mask is not None:
        a, b = a[mask], b[mask]
    if a.size == 0:
        return 0.0
    return float(np.max(np.abs(a - b)) / max(1.0, np.max(np.abs(b))))


def gpu_state_from_oracle(ost):
    """The oracle's state dict (scaled coordinates) in the library's layout; the cached
    products are left to the library (recomputed by its SpMV)."""
    return {"x": ost["x"], "x0": ost["x0"], "xsum": ost["xsum"], "y": ost["y"], "y0": ost["y0"],
            "ysum": ost["ysum"], "eta": ost["eta"], "omega": ost["omega"], "wsum": ost["wsum"],
            "phi0": ost["phi0"], "phi_prev": ost["phi_prev"],
            "comp0": [ost["comp0_rp2"], ost["comp0_rd2"], ost["comp0_gap"]],
            "attempts": int(ost["attempts"]), "accepted": int(ost["accepted"]), "k": int(ost["k"]),
            "restarts": int(ost["restarts"]), "started": int(ost["started"]), "status": int(ost["status"])}


def one_evaluation(prob, g, o):
    """Loads the oracle's current state into the library, runs one PDHG evaluation on both,
    and returns the errors of xhat, of yhat per cone role, of the next Halpern iterate and
    of the next step size (relative), with both sides' accept decisions."""
    ost = o.state()
    g.set_state(gpu_state_from_oracle(ost))
    g.run(1)
    o.run(1)
    gs, os_ = g.get_state(), o.state()
    masks = role_masks(prob)
    err = {"xhat": _rel(gs["xhat"], os_["xh"])}
    for name, mk in masks.items():
        err["yhat_" + name] = _rel(gs["yhat"], os_["yh"], mk)
    err["x"] = _rel(gs["x"], os_["x"])
    err["y"] = _rel(gs["y"], os_["y"])
    err["eta"] = abs(gs["eta"] - os_["eta"]) / os_["eta"]
    acc = (gs["accepted"] - int(ost["accepted"]), int(os_["accepted"] - ost["accepted"]))
    return err, acc

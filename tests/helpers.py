"""Shared test helpers: run the oracle and the CUDA library on the same input
and compare in particle-id space with the normalised errors

    rho:  max_a |rho - rho_ref| / rho_ref
    C:    max_a max_ij |C - C_ref| / (max_ij |C_ref| cond(tau_ref))
    a:    max_a |a - a_ref|_inf / sum_b |pair term|          (oracle's sa)
    du:   max_a |du - du_ref| / sum_b |pair term|            (oracle's sdu)
"""
import numpy as np

import oracle
import sph_inputs  # noqa: F401


def by_id(s):
    """State dict re-ordered so that index == id (the oracle's view)."""
    order = np.argsort(s["id"], kind="stable")
    return {k: (v[order] if isinstance(v, np.ndarray) else v) for k, v in s.items()}


def box_of(s):
    return oracle.Box(s["lo"], s["hi"], s["periodic"])


def oracle_params(**kw):
    p = oracle.Params()
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def oracle_outputs(s, **kw):
    s = by_id(s)
    rc, out = oracle.outputs(box_of(s), s, oracle_params(**kw))
    return rc, s, out


def sym(c6):
    c6 = np.asarray(c6)
    return np.stack([np.stack([c6[..., 0], c6[..., 1], c6[..., 2]], -1),
                     np.stack([c6[..., 1], c6[..., 3], c6[..., 4]], -1),
                     np.stack([c6[..., 2], c6[..., 4], c6[..., 5]], -1)], -2)


def field_errors(got, ref):
    """Normalised errors of every output field (got: GPU arrays by id)."""
    e = {}
    e["rho"] = float(np.max(np.abs(got["rho"] - ref["rho"]) / ref["rho"]))
    e["p"] = float(np.max(np.abs(got["p"] - ref["p"]) / np.abs(ref["p"]).clip(1e-300)))
    e["c"] = float(np.max(np.abs(got["c"] - ref["c"]) / np.abs(ref["c"]).clip(1e-300)))
    T = sym(ref["tau"])
    kappa = np.linalg.cond(T)
    cmax = np.abs(ref["iad"]).max(1)
    e["iad"] = float(np.max(np.abs(got["iad"] - ref["iad"]).max(1) / (cmax * kappa)))
    a_g = np.stack([got["ax"], got["ay"], got["az"]], 1)
    a_r = np.stack([ref["ax"], ref["ay"], ref["az"]], 1)
    sa = ref["sa"].clip(1e-300)
    e["a"] = float(np.max(np.abs(a_g - a_r).max(1) / sa))
    sdu = np.maximum(ref["sdu"], 1e-300)
    e["du"] = float(np.max(np.abs(got["du"] - ref["du"]) / sdu))
    # field-relative (reported only)
    e["a_field_rel"] = float(np.abs(a_g - a_r).max() / max(np.abs(a_r).max(), 1e-300))
    return e

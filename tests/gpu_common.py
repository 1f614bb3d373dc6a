"""Helpers shared by the GPU tests: parity metrics and grid construction."""
import numpy as np

import paper_2607_08743_gb300 as sk


def rel_err(a, b, active_only=False, g=3, floor=0.0):
    """Per-field max |a - b| / max(max |b|, floor).  `floor` keeps fields that
    vanish in the continuum solution and are non-zero only at truncation level
    (e.g. Theta in the gauge wave) from being judged relative to ~1e-12 noise;
    fields with scale 0 are compared in absolute terms."""
    if active_only:
        a = a[:, g:-g, g:-g, g:-g]
        b = b[:, g:-g, g:-g, g:-g]
    d = np.abs(a - b).max(axis=(1, 2, 3))
    s = np.maximum(np.abs(b).max(axis=(1, 2, 3)), floor)
    return np.where(s > 0, d / np.where(s > 0, s, 1.0), d)


def grid_for(patches, nlevels=1, dx0=None, **prm):
    dx0 = dx0 if dx0 is not None else patches[0].dx
    return sk.Grid(nlevels, dx0, patches, sk.Params(**prm))


def sk_params_to_oracle(prm):
    import oracle
    return oracle.Params(kappa1=prm.kappa1, kappa2=prm.kappa2, eta=prm.eta, sigma_ko=prm.sigma_ko,
                         w_floor=prm.w_floor, lapse=prm.lapse, shift=prm.shift,
                         lapse_uses_khat=prm.lapse_uses_khat)

"""Equatorial reflection symmetry (Sec. 2.2.2: evolve z >= 0 only) in the
oracle, pinned against the full domain: on data symmetric under z -> -z, the
half-domain evolution with reflected ghosts equals the upper half of the
full-domain evolution -- for a uniform patch with Sommerfeld ghosts and for
the Berger-Oliger hierarchy -- and the reflection itself against brute force."""
import numpy as np
import pytest

import initial_data as idd
import oracle


def test_reflection_fill_brute_force():
    p = idd.Patch(n=(6, 5, 4), dx=0.5, origin=(-1.0, -1.0, 0.0))
    u = np.random.default_rng(3).normal(size=p.shape)
    v = oracle.fill_zreflect(p, u)
    g = p.g
    for f in range(25):
        for k in range(g):  # ghost layer k mirrors active layer 2g - 1 - k
            assert np.array_equal(v[f, k], idd.Z_PARITY[f] * u[f, 2 * g - 1 - k])
    assert np.array_equal(v[:, g:], u[:, g:])
    with pytest.raises(ValueError):
        oracle.fill_zreflect(idd.Patch(n=(4, 4, 4), dx=0.5, origin=(0, 0, 0.5)), u[:, :, :10, :10])


def _symmetric_puncture(n=16):
    p = idd.centred_patch(n, 0.5)
    u = idd.add_noise(p, idd.punctures(p, [1.0], [(0.0, 0.0, 0.0)]), 1e-6, idd.PUNCTURE_SEED)
    return p, idd.symmetrise_z(p, u)


def test_half_domain_equals_full_domain_uniform():
    p, u = _symmetric_puncture()
    ph = idd.upper_half(p)
    uh = idd.upper_half_array(p, u)
    dt = 0.25 * p.dx
    prm = oracle.Params()
    for _ in range(2):
        u = oracle.rk4_step(p, u, dt, prm, bc=oracle.BC_SOMMERFELD)
        uh = oracle.rk4_step(ph, uh, dt, prm, bc=oracle.BC_SOMMERFELD | oracle.BC_ZREFLECT)
    g = p.g
    full_upper = idd.upper_half_array(p, u)[:, g:-g, g:-g, g:-g]
    half = uh[:, g:-g, g:-g, g:-g]
    assert np.abs(half - full_upper).max() <= 1e-14 * np.abs(full_upper).max()
    # the full-domain evolution kept the symmetry, and the reflected ghosts
    # of the half domain are its lower half
    assert np.abs(idd.symmetrise_z(p, u) - u)[:, g:-g, g:-g, g:-g].max() <= 1e-14


def test_half_domain_equals_full_domain_hierarchy():
    h = idd.small_binary(n_fixed=16, n_moving=12, n_levels=3, n_fixed_levels=2, dx0=1.0, sep=2.0)
    states = idd.hierarchy_data(h, noise=0.0)  # Brill-Lindquist on z = 0: symmetric
    hh = idd.upper_half_hierarchy(h)
    half = [idd.upper_half_array(p, u) for p, u in zip(h.patches, states)]
    full = oracle.BOHierarchy(h, states, oracle.Params(), courant=0.5)
    half_bo = oracle.BOHierarchy(hh, half, oracle.Params(), courant=0.5, zsym=True)
    full.level_step(0)
    half_bo.level_step(0)
    g = 3
    for i, p in enumerate(h.patches):
        a = idd.upper_half_array(p, full.current(i))[:, g:-g, g:-g, g:-g]
        b = half_bo.current(i)[:, g:-g, g:-g, g:-g]
        scale = np.maximum(np.abs(a).max(axis=(1, 2, 3)), 1e-300)
        err = (np.abs(a - b).max(axis=(1, 2, 3)) / scale).max()
        assert err <= 1e-12, (i, err)

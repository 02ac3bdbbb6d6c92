"""Seeded synthetic inputs for the potential-field solve.

This module only makes inputs: inner-boundary Br maps on the theta-phi grid
of cell centres, and seeded random vectors.  It holds none of the solver's
arithmetic and is shared by the tests, the oracle checks and the benchmark.

The paper measures on a magnetogram-derived Br map (Sec. 4.1) that is not
available here; ``bipole_br`` stands in for it with the same kind of
structure: a global dipole plus many small opposite-polarity Gaussian
bipoles, flux balanced over the sphere.
"""
from __future__ import annotations

import numpy as np

DEFAULT_SEED = 1709


def theta_faces(nt: int) -> np.ndarray:
    """Uniform colatitude faces j*pi/nt."""
    f = np.pi * np.arange(nt + 1) / nt
    f[0], f[-1] = 0.0, np.pi
    return f


def _centres(t_faces: np.ndarray, np_: int):
    tc = 0.5 * (t_faces[1:] + t_faces[:-1])
    dt = np.diff(t_faces)
    pc = (np.arange(np_) + 0.5) * (2.0 * np.pi / np_)
    return tc, dt, pc


def ylm_br(nt: int, np_: int, l: int = 3, m: int = 2, t_faces: np.ndarray | None = None):
    """Real spherical-harmonic Br = P_l^m(cos th) cos(m ph), scaled to unit
    peak amplitude over the sphere, sampled at the cell centres.

    Returns (br[nt, np], scale) where scale is the factor applied to
    P_l^m cos(m ph), so that an analytic solution can use the same shape."""
    from scipy.special import lpmv

    tf = theta_faces(nt) if t_faces is None else np.asarray(t_faces, dtype=np.float64)
    tc, _, pc = _centres(tf, np_)
    fine = np.cos(np.linspace(0.0, np.pi, 200001))
    peak = np.max(np.abs(lpmv(m, l, fine)))
    scale = 1.0 / peak
    br = scale * lpmv(m, l, np.cos(tc))[:, None] * np.cos(m * pc)[None, :]
    return np.ascontiguousarray(br), scale


def ylm_shape(l: int, m: int, theta: np.ndarray, phi: np.ndarray, scale: float) -> np.ndarray:
    """The same angular shape as ``ylm_br`` evaluated at arbitrary points."""
    from scipy.special import lpmv

    return scale * lpmv(m, l, np.cos(theta)) * np.cos(m * phi)


def _unit(theta, phi):
    theta, phi = np.broadcast_arrays(np.asarray(theta, dtype=np.float64),
                                     np.asarray(phi, dtype=np.float64))
    st = np.sin(theta)
    return np.stack([st * np.cos(phi), st * np.sin(phi), np.cos(theta)], axis=-1)


def bipole_br(nt: int, np_: int, seed: int = DEFAULT_SEED, n_bipoles: int = 200,
              dipole_g: float = 5.0, width_deg=(0.5, 3.0), amp_g=(1.0, 1000.0),
              sep_over_width: float = 2.5, t_faces: np.ndarray | None = None) -> np.ndarray:
    """Flux-balanced synthetic magnetogram Br[nt, np] (gauss).

    Dipole B0 cos(th) plus ``n_bipoles`` pairs of opposite-sign Gaussians
    exp(-d^2 / w^2) in great-circle angle d.  Bipole centres are uniform on the
    sphere, widths w uniform in ``width_deg``, amplitudes log-uniform in
    ``amp_g``, pole separation ``sep_over_width`` * w, tilt uniform in
    [0, 2 pi).  Finally the discrete area-weighted mean
    sum(Br sin th dth dph) / sum(sin th dth dph) is subtracted so the net
    flux through the cells is zero to rounding.  Deterministic in ``seed``.
    """
    rng = np.random.default_rng(seed)
    tf = theta_faces(nt) if t_faces is None else np.asarray(t_faces, dtype=np.float64)
    tc, dt, pc = _centres(tf, np_)
    x = _unit(tc[:, None], pc[None, :])  # [nt, np, 3]
    br = dipole_g * np.cos(tc)[:, None] * np.ones((1, np_))
    # draw every bipole's parameters first, in a fixed order
    ct = rng.uniform(-1.0, 1.0, n_bipoles)
    phc = rng.uniform(0.0, 2.0 * np.pi, n_bipoles)
    w = np.deg2rad(rng.uniform(width_deg[0], width_deg[1], n_bipoles))
    amp = np.exp(rng.uniform(np.log(amp_g[0]), np.log(amp_g[1]), n_bipoles))
    tilt = rng.uniform(0.0, 2.0 * np.pi, n_bipoles)
    thc = np.arccos(ct)
    for b in range(n_bipoles):
        c = _unit(thc[b], phc[b])
        # local north (towards decreasing theta) and east unit vectors at c
        north = -np.array([np.cos(thc[b]) * np.cos(phc[b]), np.cos(thc[b]) * np.sin(phc[b]),
                           -np.sin(thc[b])])
        east = np.array([-np.sin(phc[b]), np.cos(phc[b]), 0.0])
        u = np.cos(tilt[b]) * north + np.sin(tilt[b]) * east
        half = 0.5 * sep_over_width * w[b]
        for sign in (1.0, -1.0):
            pole = np.cos(half) * c + sign * np.sin(half) * u
            dotp = np.clip(x @ pole, -1.0, 1.0)
            crs = np.linalg.norm(np.cross(x, pole), axis=-1)
            d = np.arctan2(crs, dotp)
            br += sign * amp[b] * np.exp(-(d / w[b]) ** 2)
    area = (np.sin(tc) * dt)[:, None] * np.full((1, np_), 2.0 * np.pi / np_)
    br -= np.sum(br * area) / np.sum(area)
    return np.ascontiguousarray(br)


def random_field(shape, seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """Seeded uniform random array (test vectors for operator probes)."""
    return np.random.default_rng(seed).uniform(lo, hi, size=shape)

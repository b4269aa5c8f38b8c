"""Equilibration-ratio analysis of Sec. III on top of the library's S(k).

* ER_m(|k|) = S_m^num(|k|) / S_m^th(|k|) (Eq. er_of_k), S_m from
  flbm_structure_factor averaged over snapshots, S_m^th the flat lattice
  theory value per node: 3, 3, 5, 1 times rho0 kT for rho, sum_a rho u_a,
  sum_a Pi_aa, sum_{a<b} Pi_ab and rho0 kT for each momentum component (the
  lattice ideal-gas invariant measure <dg_i dg_j> = (rho0 kT / c_s^2) w_i
  delta_ij).
* The min/max of ER_m over the shells |n| in [4, 64] (Fig. 2), shells being
  integer wavevector radii round(|n|).

The per-snapshot ratio comes from the C ABI (flbm_spectral_er: the CUDA
path's cuFFT spectrum and FP64 shell sums over S_m^th); here the snapshots
are averaged and the window extrema taken.
"""
from __future__ import annotations

import numpy as np

from . import flbm

THEORY_FACTOR = {
    flbm.FLBM_OBS_RHO: 3.0,
    flbm.FLBM_OBS_JSUM: 3.0,
    flbm.FLBM_OBS_PI_DIAG: 5.0,
    flbm.FLBM_OBS_PI_OFFDIAG: 1.0,
    flbm.FLBM_OBS_JX: 1.0,
    flbm.FLBM_OBS_JY: 1.0,
    flbm.FLBM_OBS_JZ: 1.0,
}
PAPER_OBSERVABLES = (flbm.FLBM_OBS_RHO, flbm.FLBM_OBS_JSUM, flbm.FLBM_OBS_PI_DIAG,
                     flbm.FLBM_OBS_PI_OFFDIAG)


def theory(observable: int, rho0: float, kT: float) -> float:
    """Flat S_m^th of one observable (per-node equilibrium variance)."""
    return THEORY_FACTOR[observable] * rho0 * kT


def er_spectrum(lat, nshell: int, snapshots: int, every: int,
                observables=PAPER_OBSERVABLES):
    """Advance `lat` by `every` steps `snapshots` times and return
    {observable: (ER_m per shell, shell populations)} of the snapshot average."""
    acc = {m: np.zeros(nshell) for m in observables}
    cnt = {}
    for _ in range(snapshots):
        lat.step(every)
        for m in observables:
            er, c = lat.spectral_er(m, nshell)
            acc[m] += er
            cnt[m] = c
    return {m: (acc[m] / snapshots, cnt[m]) for m in observables}


def window_extrema(er, counts, kmin: int = 4, kmax: int = 64):
    """(min, max) of ER_m over the populated shells kmin <= |n| <= kmax."""
    idx = [s for s in range(len(er)) if kmin <= s <= kmax and counts[s] > 0]
    if not idx:
        return float("nan"), float("nan")
    v = np.asarray(er)[idx]
    return float(v.min()), float(v.max())

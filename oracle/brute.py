"""Visible normals by brute-force ray casting: an oracle independent of every formula.

Sec. 2 ("Definition") defines the GGX VNDF as the distribution of the normals
found where parallel rays, arriving from direction wi, first hit a truncated
ellipsoid.  M = diag(1/ax, 1/ay, 1) maps the unit hemisphere onto it, so its
semi-axes are (1/ax, 1/ay, 1): ax^2 x^2 + ay^2 y^2 + z^2 = 1, z >= 0.  This module
casts such rays and records those normals.  It uses none of the paper's
sampling formulas, densities or transformations, so agreement with the
sampler is a check of the whole construction.

Test infrastructure only; shares no code with the CUDA path.
"""
import numpy as np


def _orthonormal_frame(wi):
    w = np.asarray(wi, dtype=np.float64)
    w = w / np.linalg.norm(w)
    helper = np.array([1.0, 0.0, 0.0]) if abs(w[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    e1 = np.cross(w, helper)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(w, e1)
    return w, e1, e2


def visible_normals(wi, ax, ay, n_rays, rng):
    """Normals at the first hits of n_rays parallel rays with direction -wi.

    Ray origins are uniform on a disk perpendicular to wi that covers the
    projection of the ellipsoid; rays that miss, or whose first hit lies on
    the removed lower half (z < 0), are discarded.  Returns an array (3, K).
    """
    w, e1, e2 = _orthonormal_frame(wi)
    radius = max(1.0 / ax, 1.0 / ay, 1.0) * 1.01
    r = radius * np.sqrt(rng.random(n_rays))
    t = 2.0 * np.pi * rng.random(n_rays)
    # origins far out along +wi, offset within the disk
    o = (2.0 * radius * w)[:, None] + e1[:, None] * (r * np.cos(t)) + e2[:, None] * (r * np.sin(t))
    d = -w[:, None] * np.ones(n_rays)
    # ellipsoid as the quadric p^T A p = 1 with A = diag(ax^2, ay^2, 1)
    a_diag = np.array([ax ** 2, ay ** 2, 1.0])[:, None]
    qa = (a_diag * d * d).sum(0)
    qb = 2.0 * (a_diag * o * d).sum(0)
    qc = (a_diag * o * o).sum(0) - 1.0
    disc = qb * qb - 4.0 * qa * qc
    hit = disc > 0.0
    t_near = (-qb - np.sqrt(np.where(hit, disc, 0.0))) / (2.0 * qa)
    p = o + d * t_near
    keep = hit & (p[2] >= 0.0)
    p = p[:, keep]
    nrm = a_diag * p  # gradient of the quadric
    return nrm / np.linalg.norm(nrm, axis=0)

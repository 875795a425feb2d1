"""Seeded synthetic inputs for the VNDF workloads (shared by the oracle tests and the GPU path).

This module only draws input data: incident directions, roughness values,
per-query sample counts and auxiliary vectors, with the distributions of the
five workloads below.  It holds none of the sampling method's arithmetic and
imports neither the oracle nor the CUDA library.  The uniforms (u1, u2) that the
method itself consumes are not drawn here: each side produces them with its own
Philox4x32-10 implementation.

Every generator takes (seed, device) and returns contiguous float32 (or int32)
torch tensors on that device, so the large workloads can be drawn directly in
device memory.  Draws are made in float64 and rounded once to float32.

Workloads (sizes are the defaults):
* ``isotropic_2e20``   2^20 samples, isotropic alpha ~ U[0.01, 1],
                       wi uniform on the upper hemisphere (cos ~ U[0, 1)).
* ``anisotropic_stream``  2^28 samples, alpha_x, alpha_y ~ log-U[1e-3, 1]
                       independently, cos(theta_i) ~ U[1e-4, 1], phi ~ U[0, 2 pi).
* ``albedo_grid``      4096 queries: 64 cos(theta_i) = linspace(0.01, 1) x 64
                       alpha = geomspace(1e-3, 1) (isotropic), wi in the xz plane,
                       per-query counts floor(256 * 256^r), r ~ U[0, 1), in [256, 65536].
* ``adjoint_2e24``     2^24 samples, alpha ~ log-U[1e-2, 1], cos(theta_i) ~ U[0.05, 1],
                       plus random unit vectors c (normalised Gaussians) for the loss.
* ``roughness_map``    256 x 256 texels, alpha_x, alpha_y ~ U[0.05, 0.8],
                       cos(theta_i) ~ U[0.1, 1] per texel, and a smooth target
                       field of unit vectors.
* ``sphere_stream``    2^28 samples for the extended domain: wi uniform on the
                       whole sphere (cos(theta_i) ~ U[-1, 1], half of them below
                       the horizon), alpha_x, alpha_y ~ log-U[1e-3, 1].
* ``hemisphere_stream`` 2^28 directions for the stand-alone hemisphere sampler:
                       uniform on the whole sphere, lengths ~ log-U[0.5, 2].
* ``wide_stream``      stress inputs for the tests: wi uniform on the whole sphere
                       with lengths ~ log-U[1e-3, 1e3], alpha_x, alpha_y ~
                       log-U[1e-5, 10] independently, and explicit uniforms on the
                       2^-24 grid of [0, 1) with 1 % of them set to the ends and
                       quarter points (0, 2^-24, 1/4, 1/2, 3/4, 1 - 2^-24).
"""
import math

import torch


def _gen(seed, device):
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def _uniform(g, n, lo, hi, device):
    return lo + (hi - lo) * torch.rand(n, generator=g, dtype=torch.float64, device=device)


def _log_uniform(g, n, lo, hi, device):
    return torch.exp(_uniform(g, n, math.log(lo), math.log(hi), device))


def _directions(g, n, cos_lo, cos_hi, device):
    """Unit vectors with cos(theta) ~ U[cos_lo, cos_hi] and phi ~ U[0, 2 pi)."""
    ct = _uniform(g, n, cos_lo, cos_hi, device)
    phi = _uniform(g, n, 0.0, 2.0 * math.pi, device)
    st = torch.sqrt(torch.clamp(1.0 - ct * ct, min=0.0))
    return st * torch.cos(phi), st * torch.sin(phi), ct


def _f32(*ts):
    return tuple(t.to(torch.float32).contiguous() for t in ts)


def isotropic_2e20(n=1 << 20, seed=11, device="cpu"):
    g = _gen(seed, device)
    wx, wy, wz = _directions(g, n, 0.0, 1.0, device)
    alpha = _uniform(g, n, 0.01, 1.0, device)
    wx, wy, wz, alpha = _f32(wx, wy, wz, alpha)
    return {"wi_x": wx, "wi_y": wy, "wi_z": wz, "alpha_x": alpha}


def anisotropic_stream(n=1 << 28, seed=12, device="cpu"):
    g = _gen(seed, device)
    wx, wy, wz = _directions(g, n, 1e-4, 1.0, device)
    ax = _log_uniform(g, n, 1e-3, 1.0, device)
    ay = _log_uniform(g, n, 1e-3, 1.0, device)
    wx, wy, wz, ax, ay = _f32(wx, wy, wz, ax, ay)
    return {"wi_x": wx, "wi_y": wy, "wi_z": wz, "alpha_x": ax, "alpha_y": ay}


def albedo_grid(n_cos=64, n_alpha=64, seed=3, device="cpu", min_count=256, max_count=65536):
    cos_t = torch.linspace(0.01, 1.0, n_cos, dtype=torch.float64, device=device)
    alpha = torch.exp(torch.linspace(math.log(1e-3), 0.0, n_alpha, dtype=torch.float64, device=device))
    ct, al = torch.meshgrid(cos_t, alpha, indexing="ij")
    ct = ct.reshape(-1)
    al = al.reshape(-1)
    st = torch.sqrt(torch.clamp(1.0 - ct * ct, min=0.0))
    g = _gen(seed, device)
    r = torch.rand(ct.numel(), generator=g, dtype=torch.float64, device=device)
    counts = torch.floor(float(min_count) * (float(max_count) / min_count) ** r)
    counts = torch.clamp(counts, min_count, max_count).to(torch.int32).contiguous()
    wx, wy, wz, al = _f32(st, torch.zeros_like(st), ct, al)
    return {"wi_x": wx, "wi_y": wy, "wi_z": wz, "alpha_x": al, "n_samples": counts}


def adjoint_2e24(n=1 << 24, seed=4, device="cpu"):
    g = _gen(seed, device)
    wx, wy, wz = _directions(g, n, 0.05, 1.0, device)
    ax = _log_uniform(g, n, 1e-2, 1.0, device)
    ay = _log_uniform(g, n, 1e-2, 1.0, device)
    c = torch.randn(3, n, generator=g, dtype=torch.float64, device=device)
    c = c / torch.linalg.vector_norm(c, dim=0, keepdim=True)
    wx, wy, wz, ax, ay, cx, cy, cz = _f32(wx, wy, wz, ax, ay, c[0], c[1], c[2])
    return {"wi_x": wx, "wi_y": wy, "wi_z": wz, "alpha_x": ax, "alpha_y": ay,
            "c_x": cx, "c_y": cy, "c_z": cz}


def roughness_map(res=256, seed=5, device="cpu"):
    g = _gen(seed, device)
    t = res * res
    ax = _uniform(g, t, 0.05, 0.8, device)
    ay = _uniform(g, t, 0.05, 0.8, device)
    wx, wy, wz = _directions(g, t, 0.1, 1.0, device)
    # smooth target field of unit vectors tilted up to ~0.3 rad from the pole
    yy, xx = torch.meshgrid(torch.arange(res, dtype=torch.float64, device=device),
                            torch.arange(res, dtype=torch.float64, device=device), indexing="ij")
    a = 0.15 * torch.sin(2.0 * math.pi * xx / res).reshape(-1)
    b = 0.15 * torch.cos(2.0 * math.pi * yy / res).reshape(-1)
    n = torch.sqrt(1.0 + a * a + b * b)
    ax, ay, wx, wy, wz, tx, ty, tz = _f32(ax, ay, wx, wy, wz, a / n, b / n, 1.0 / n)
    return {"alpha_x": ax, "alpha_y": ay, "wi_x": wx, "wi_y": wy, "wi_z": wz,
            "target_x": tx, "target_y": ty, "target_z": tz}


def sphere_stream(n=1 << 28, seed=13, device="cpu"):
    g = _gen(seed, device)
    wx, wy, wz = _directions(g, n, -1.0, 1.0, device)
    ax = _log_uniform(g, n, 1e-3, 1.0, device)
    ay = _log_uniform(g, n, 1e-3, 1.0, device)
    wx, wy, wz, ax, ay = _f32(wx, wy, wz, ax, ay)
    return {"wi_x": wx, "wi_y": wy, "wi_z": wz, "alpha_x": ax, "alpha_y": ay}


def hemisphere_stream(n=1 << 28, seed=14, device="cpu"):
    g = _gen(seed, device)
    wx, wy, wz = _directions(g, n, -1.0, 1.0, device)
    r = _log_uniform(g, n, 0.5, 2.0, device)
    wx, wy, wz = _f32(wx * r, wy * r, wz * r)
    return {"wi_x": wx, "wi_y": wy, "wi_z": wz}


def wide_stream(n=1 << 16, seed=15, device="cpu"):
    g = _gen(seed, device)
    wx, wy, wz = _directions(g, n, -1.0, 1.0, device)
    r = _log_uniform(g, n, 1e-3, 1e3, device)
    ax = _log_uniform(g, n, 1e-5, 10.0, device)
    ay = _log_uniform(g, n, 1e-5, 10.0, device)
    k = torch.floor(torch.rand(2, n, generator=g, dtype=torch.float64, device=device) * 2.0 ** 24)
    u = k * 2.0 ** -24
    special = torch.tensor([0.0, 2.0 ** -24, 0.25, 0.5, 0.75, 1.0 - 2.0 ** -24], dtype=torch.float64, device=device)
    pick = torch.rand(2, n, generator=g, dtype=torch.float64, device=device) < 0.01
    which = torch.randint(0, special.numel(), (2, n), generator=g, device=device)
    u = torch.where(pick, special[which], u)
    wx, wy, wz, ax, ay, u1, u2 = _f32(wx * r, wy * r, wz * r, ax, ay, u[0], u[1])
    return {"wi_x": wx, "wi_y": wy, "wi_z": wz, "alpha_x": ax, "alpha_y": ay, "u1": u1, "u2": u2}

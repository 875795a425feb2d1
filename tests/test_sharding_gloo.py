"""Multi-rank path on CPU: world_size 2 over gloo (no GPU).

Each rank evaluates the oracle on its own shard with the counter or stream
base that sharding.py assigns; rank 0 gathers and checks that the shards
concatenate bit-for-bit to a single-process run, and that the timing
reduction returns the maximum over ranks.  The CUDA kernels use the same
counter layout, so this is the property that makes multi-GPU runs need no
data-path collective.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2306_05044_gb300 import sharding

N_PER_RANK = 3001
N_QUERIES = 7


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import sys
        root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
        sys.path.insert(0, root)
        import workloads
        from oracle import microfacet, philox, vndf

        # samples: weak scaling over one global index range
        base, n = sharding.sample_shard(rank, world, N_PER_RANK)
        d = workloads.anisotropic_stream(n=world * N_PER_RANK, seed=21)
        sl = slice(base, base + n)
        wi = np.stack([d[k][sl].numpy() for k in ("wi_x", "wi_y", "wi_z")])
        u1, u2 = philox.sample_uniforms(2, base, 0, n)
        wm, pdf = vndf.sample_vndf_with_pdf(u1, u2, wi, d["alpha_x"][sl].numpy(), d["alpha_y"][sl].numpy())
        local = torch.from_numpy(np.concatenate([wm, pdf[None]]))
        gathered = [torch.empty_like(local) for _ in range(world)]
        dist.all_gather(gathered, local)
        # albedo: queries split, stream base = first query of the shard
        g = workloads.albedo_grid(n_cos=7, n_alpha=1, seed=3, max_count=600)
        q0, q1 = sharding.query_shard(rank, world, N_QUERIES)
        wi_q = np.stack([g[k].numpy()[q0:q1] for k in ("wi_x", "wi_y", "wi_z")])
        a = g["alpha_x"].numpy()[q0:q1]
        e = microfacet.albedo_estimate(wi_q, a, a, g["n_samples"].numpy()[q0:q1], 0.04, seed=3, stream_base=q0)
        counts = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(counts, torch.tensor([q1 - q0]))
        padded = torch.zeros(N_QUERIES, dtype=torch.float64)
        padded[: q1 - q0] = torch.from_numpy(e)
        parts = [torch.empty_like(padded) for _ in range(world)]
        dist.all_gather(parts, padded)
        # fitting: texels split, stream base = first texel; the loss shares are summed over ranks
        from oracle import fit as ofit
        m = workloads.roughness_map(res=FIT_RES, seed=5)
        t0, t1 = sharding.texel_shard(rank, world, FIT_RES * FIT_RES)
        st, wi_t, tg = _fit_inputs(m, t0, t1)
        losses = []
        for step in (1, 2):
            st, loss, _ = ofit.fit_step(st, wi_t, tg, FIT_SAMPLES, step, seed=7, stream_base=t0,
                                        n_total=FIT_RES * FIT_RES)
            losses.append(sharding.sum_over_ranks(loss))
        ax_parts = [torch.zeros(FIT_RES * FIT_RES, dtype=torch.float64) for _ in range(world)]
        ax_local = torch.zeros(FIT_RES * FIT_RES, dtype=torch.float64)
        ax_local[: t1 - t0] = torch.from_numpy(st["ax"])
        dist.all_gather(ax_parts, ax_local)
        tcounts = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(tcounts, torch.tensor([t1 - t0]))
        # timing reduction
        t_max = sharding.max_over_ranks(1.0 + rank)
        if rank == 0:
            torch.save({"samples": torch.cat(gathered, dim=1),
                        "albedo": torch.cat([p[: int(c.item())] for p, c in zip(parts, counts)]),
                        "fit_ax": torch.cat([p[: int(c.item())] for p, c in zip(ax_parts, tcounts)]),
                        "fit_losses": losses, "t_max": t_max}, os.path.join(out_dir, "result.pt"))
    finally:
        dist.destroy_process_group()


FIT_RES, FIT_SAMPLES = 3, 16


def _fit_inputs(m, t0, t1):
    st = {"ax": m["alpha_x"].numpy()[t0:t1].astype(np.float64), "ay": m["alpha_y"].numpy()[t0:t1].astype(np.float64)}
    st.update({k: np.zeros(t1 - t0) for k in ("mx", "my", "vx", "vy")})
    wi = np.stack([m[k].numpy()[t0:t1] for k in ("wi_x", "wi_y", "wi_z")]).astype(np.float64)
    tg = np.stack([m[k].numpy()[t0:t1] for k in ("target_x", "target_y", "target_z")]).astype(np.float64)
    return st, wi, tg


def test_shards_concatenate_to_single_run(tmp_path):
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = torch.load(os.path.join(tmp_path, "result.pt"))
    import workloads
    from oracle import microfacet, philox, vndf
    n = world * N_PER_RANK
    d = workloads.anisotropic_stream(n=n, seed=21)
    wi = np.stack([d[k].numpy() for k in ("wi_x", "wi_y", "wi_z")])
    u1, u2 = philox.sample_uniforms(2, 0, 0, n)
    wm, pdf = vndf.sample_vndf_with_pdf(u1, u2, wi, d["alpha_x"].numpy(), d["alpha_y"].numpy())
    np.testing.assert_array_equal(res["samples"].numpy(), np.concatenate([wm, pdf[None]]))
    g = workloads.albedo_grid(n_cos=7, n_alpha=1, seed=3, max_count=600)
    wi_q = np.stack([g[k].numpy() for k in ("wi_x", "wi_y", "wi_z")])
    a = g["alpha_x"].numpy()
    e = microfacet.albedo_estimate(wi_q, a, a, g["n_samples"].numpy(), 0.04, seed=3)
    np.testing.assert_array_equal(res["albedo"].numpy(), e)
    from oracle import fit as ofit
    m = workloads.roughness_map(res=FIT_RES, seed=5)
    st, wi_t, tg = _fit_inputs(m, 0, FIT_RES * FIT_RES)
    for step in (1, 2):
        st, loss, _ = ofit.fit_step(st, wi_t, tg, FIT_SAMPLES, step, seed=7)
        assert abs(res["fit_losses"][step - 1] / loss - 1) < 1e-12
    np.testing.assert_array_equal(res["fit_ax"].numpy(), st["ax"])
    assert res["t_max"] == 2.0


def test_shard_arithmetic():
    for world in (1, 2, 3, 8):
        ranges = [sharding.query_shard(r, world, 4096) for r in range(world)]
        assert ranges[0][0] == 0 and ranges[-1][1] == 4096
        assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
        assert max(b - a for a, b in ranges) - min(b - a for a, b in ranges) <= 1
        bases = [sharding.sample_shard(r, world, 1 << 28)[0] for r in range(world)]
        assert bases == [r << 28 for r in range(world)]
    with pytest.raises(ValueError):
        sharding.sample_shard(2, 2, 10)
    assert sharding.max_over_ranks(3.5) == 3.5

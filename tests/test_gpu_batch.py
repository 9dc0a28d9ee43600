"""Batched total viewsheds (several DEMs per launch) and prepared batches
replayed from a CUDA graph, against the single-DEM path."""
import numpy as np
import pytest

import paper_2003_02200_gb300 as tvs
from paper_2003_02200_gb300 import terrain

pytestmark = pytest.mark.gpu

# Per-cell totals are exact sums of FP32 group sums (8 directions each), so a
# batch gives bit for bit what the single-DEM path gives whenever its chunk
# cuts fall on group boundaries (always here: 8 directions of every job fit
# each budget below).


def _jobs(specs, seed=0):
    import torch
    jobs = []
    for i, (rows, cols, n, step, h0, rng) in enumerate(specs):
        dem = terrain.fractal_dem(rows, cols, 0.6 + 0.05 * (i % 5), 300.0 + 100.0 * i, seed + i)
        d = torch.from_numpy(dem).cuda()
        jobs.append(dict(dem=d, out=torch.full_like(d, -1.0), step_m=step, obs_height_m=h0, n_sectors=n,
                         max_range_m=rng))
    return jobs


SPECS = [(40, 60, 36, 10.0, 1.5, 0.0), (130, 97, 45, 5.0, 12.0, 0.0), (64, 64, 180, 30.0, 2.0, 600.0),
         (300, 210, 24, 10.0, 1.5, 0.0), (2, 500, 8, 10.0, 3.0, 0.0), (257, 3, 16, 10.0, 1.0, 0.0),
         (90, 90, 90, 10.0, 25.0, 900.0)]


def _singles(ctx, jobs):
    import torch
    res = []
    for j in jobs:
        out = torch.empty_like(j["dem"])
        ctx.total_viewshed_device(j["dem"], j["step_m"], j["obs_height_m"], j["n_sectors"], j["max_range_m"], out=out)
        res.append(out)
    torch.cuda.synchronize()
    return [r.cpu().numpy() for r in res]


@pytest.fixture(scope="module")
def ctx():
    c = tvs.Context(0)
    yield c
    c.close()


def test_batch_matches_single_dem_path(ctx):
    import torch
    jobs = _jobs(SPECS)
    want = _singles(ctx, jobs)
    ctx.total_viewshed_batch(jobs)
    torch.cuda.synchronize()
    for j, w in zip(jobs, want):
        np.testing.assert_array_equal(j["out"].cpu().numpy(), w)


def test_batch_under_a_small_budget_spans_chunks(ctx):
    import torch
    jobs = _jobs(SPECS, seed=10)
    want = _singles(ctx, jobs)
    with tvs.Context(0, hbm_budget_bytes=40 << 20) as small:
        small.total_viewshed_batch(jobs)
    torch.cuda.synchronize()
    for j, w in zip(jobs, want):
        np.testing.assert_array_equal(j["out"].cpu().numpy(), w)


def test_prepared_batch_graph_replays(ctx):
    import torch
    jobs = _jobs(SPECS, seed=20)
    want = _singles(ctx, jobs)
    b = ctx.prepare_batch(jobs)
    info = b.info()
    assert info["jobs"] == len(jobs) and info["chunks"] >= 1 and info["kernels_per_launch"] >= 4
    assert info["evals"] == sum(tvs.count_evals(j["dem"].shape[0], j["dem"].shape[1], j["n_sectors"], j["step_m"],
                                                j["max_range_m"]) for j in jobs)
    for _ in range(2):
        for j in jobs:
            j["out"].fill_(-1.0)
        b.launch()
        torch.cuda.synchronize()
        for j, w in zip(jobs, want):
            np.testing.assert_array_equal(j["out"].cpu().numpy(), w)
    # new elevations in the same buffer are picked up by the next replay
    fresh = terrain.fractal_dem(jobs[0]["dem"].shape[0], jobs[0]["dem"].shape[1], 0.75, 700.0, seed=99)
    jobs[0]["dem"].copy_(torch.from_numpy(fresh))
    b.launch()
    torch.cuda.synchronize()
    out2 = torch.empty_like(jobs[0]["dem"])
    ctx.total_viewshed_device(jobs[0]["dem"], jobs[0]["step_m"], jobs[0]["obs_height_m"], jobs[0]["n_sectors"],
                              jobs[0]["max_range_m"], out=out2)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(jobs[0]["out"].cpu().numpy(), out2.cpu().numpy())
    assert not np.allclose(out2.cpu().numpy(), want[0])
    b.close()


def test_batch_reports_the_bad_job(ctx):
    import torch
    jobs = _jobs(SPECS[:3])
    jobs[2]["step_m"] = 0.0
    with pytest.raises(tvs.TvsError) as ei:
        ctx.total_viewshed_batch(jobs)
    assert ei.value.code == tvs._binding.TVS_ERR_ARG and "job 2" in str(ei.value)
    torch.cuda.synchronize()


def test_autotune_keeps_results_and_sets_the_handle(ctx):
    import torch
    jobs = _jobs(SPECS[:4], seed=30)
    want = _singles(ctx, jobs)
    with tvs.Context(0) as tuned:
        best, ms = tuned.autotune(jobs)
        assert ms > 0 and best == tuned.get_tuning()
        assert best["small_pov_below_w"] >= 0 and 0 <= best["sweep_max_warps"] <= 16
        for j in jobs:
            j["out"].fill_(-1.0)
        tuned.total_viewshed_batch(jobs)
        torch.cuda.synchronize()
    for j, w in zip(jobs, want):
        np.testing.assert_array_equal(j["out"].cpu().numpy(), w)


@pytest.mark.parametrize("pov_below,p4_cost", [(0, 1 << 20), (1 << 30, 107), (0, 100), (0, 130)])
def test_group_size_choice_does_not_change_results(ctx, pov_below, p4_cost):
    """Every row on 8-POV groups (4-POV cost prohibitive), every row on 4-POV
    groups (threshold huge), or a per-row mix: the per-sample measures are
    exact integers either way."""
    import torch
    jobs = _jobs(SPECS[:3], seed=40)
    want = _singles(ctx, jobs)
    with tvs.Context(0) as c:
        c.set_tuning(small_pov_below_w=pov_below, p4_cost_pct=p4_cost)
        assert c.get_tuning()["p4_cost_pct"] == p4_cost
        for j in jobs:
            c.total_viewshed_device(j["dem"], j["step_m"], j["obs_height_m"], j["n_sectors"], j["max_range_m"],
                                    out=j["out"])
        torch.cuda.synchronize()
    for j, w in zip(jobs, want):
        np.testing.assert_array_equal(j["out"].cpu().numpy(), w)

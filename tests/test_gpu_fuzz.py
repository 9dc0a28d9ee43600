"""Seeded random cases across shapes, direction counts, ranges, observer
heights and terrains: certified decisions against the FP64 oracle, FP32
decisions against the oracle's FP32-decision mode, and pruning on/off and
batched/single bit for bit."""
import numpy as np
import pytest

import paper_2003_02200_gb300 as tvs
from paper_2003_02200_gb300 import terrain

pytestmark = pytest.mark.gpu

FP32_RTOL = 4e-6


def _case(seed):
    rng = np.random.default_rng(20030220 + seed)
    kind = rng.choice(["fractal", "noise", "steps", "strip"])
    if kind == "strip":
        rows, cols = (2, int(rng.integers(3, 400))) if rng.random() < 0.5 else (int(rng.integers(3, 400)), 2)
    else:
        rows, cols = int(rng.integers(2, 130)), int(rng.integers(2, 130))
    if kind == "fractal" and min(rows, cols) >= 4:
        dem = terrain.fractal_dem(rows, cols, float(rng.uniform(0.5, 0.95)), float(rng.uniform(10, 900)),
                                  seed=int(rng.integers(1 << 30)))
    elif kind == "steps":
        dem = np.round(rng.random((rows, cols)) * 4).astype(np.float32) * 10.0 - 5.0
    else:
        dem = (rng.random((rows, cols)) * float(rng.uniform(1, 300))).astype(np.float32)
    n = int(rng.choice([1, 2, 3, 4, 7, 16, 45, 90, 180, 257]))
    h0 = float(rng.choice([0.0, 1.5, 12.0]))
    rng_m = float(rng.choice([0.0, 0.0, 35.0, 400.0]))
    step = float(rng.choice([1.0, 10.0, 30.0]))
    return dem, step, h0, n, rng_m


@pytest.fixture(scope="module")
def ctx():
    c = tvs.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("seed", range(24))
def test_fuzz_against_the_oracle_and_modes(ctx, orc, seed):
    import torch
    dem, step, h0, n, rng_m = _case(seed)
    got = ctx.total_viewshed(dem, step, h0, n, rng_m)
    o64 = orc.total_viewshed(dem, step, h0, n, rng_m, prec=64)
    np.testing.assert_allclose(got, o64, rtol=FP32_RTOL, atol=0)
    o32 = orc.total_viewshed(dem, step, h0, n, rng_m, prec=32)
    with tvs.Context(0) as c2:
        c2.set_tuning(prune=0)
        assert np.array_equal(c2.total_viewshed(dem, step, h0, n, rng_m), got)
        c2.set_tuning(fp32_decisions=1)
        np.testing.assert_allclose(c2.total_viewshed(dem, step, h0, n, rng_m), o32, rtol=FP32_RTOL, atol=0)
    d = torch.from_numpy(dem).cuda()
    other = torch.from_numpy(np.ascontiguousarray(dem[::-1, ::-1])).cuda()
    jobs = [dict(dem=d, out=torch.empty_like(d), step_m=step, obs_height_m=h0, n_sectors=n, max_range_m=rng_m),
            dict(dem=other, out=torch.empty_like(other), step_m=step, obs_height_m=h0, n_sectors=n,
                 max_range_m=rng_m)]
    ctx.total_viewshed_batch(jobs)
    torch.cuda.synchronize()
    assert np.array_equal(jobs[0]["out"].cpu().numpy(), got)

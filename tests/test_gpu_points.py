"""Singular and multiple viewsheds of a list of POVs (tvs_viewshed_points):
the sDEM mode gives the total viewshed map's value at each cell bit for bit,
the direct mode (Alg. 1-3, lines through the cell itself) matches the
oracle's definition -- with certified decisions (the default) the FP64
definition, with FP32 decisions the oracle's FP32-decision mode."""
import numpy as np
import pytest

import paper_2003_02200_gb300 as tvs
from paper_2003_02200_gb300 import terrain
from paper_2003_02200_gb300._binding import TVS_ERR_ARG

pytestmark = pytest.mark.gpu

FP32_RTOL = 4e-6


@pytest.fixture(scope="module")
def ctx():
    """Certified decisions (the library default)."""
    c = tvs.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def ctx32():
    """FP32 decisions."""
    c = tvs.Context(0)
    c.set_tuning(fp32_decisions=1)
    yield c
    c.close()


def _povs(rows, cols, count, seed):
    rng = np.random.default_rng(seed)
    p = np.stack([rng.integers(0, rows, count), rng.integers(0, cols, count)], 1)
    corners = np.array([[0, 0], [0, cols - 1], [rows - 1, 0], [rows - 1, cols - 1], [rows // 2, 0]])
    return np.concatenate([p, corners]).astype(np.int32)


# walks around multiples of the warp walk's chunk: 2 x 65 and 33 x 64 strips,
# a range of exactly 32 steps; and the longest rows (16384 samples: a 64 KB
# table of 1/d in shared memory)
@pytest.mark.parametrize("rows,cols,n,rng,h0", [(120, 90, 180, 0.0, 1.5), (64, 200, 36, 900.0, 10.0),
                                                (3, 257, 16, 0.0, 1.0), (150, 150, 45, 0.0, 0.0),
                                                (2, 65, 1, 0.0, 1.5), (33, 64, 4, 320.0, 2.0),
                                                (97, 33, 8, 0.0, 3.0), (3, 16384, 4, 0.0, 1.5)])
def test_sdem_points_equal_the_total_map(ctx, ctx32, rows, cols, n, rng, h0):
    import torch
    dem = terrain.fractal_dem(rows, cols, 0.8, 600.0, seed=rows + cols)
    d = torch.from_numpy(dem).cuda()
    povs = _povs(rows, cols, 40, seed=n)
    for c in (ctx, ctx32):
        full = c.total_viewshed_device(d, 10.0, h0, n, rng)
        got = c.viewshed_points(d, 10.0, h0, n, rng, povs, mode="sdem")
        torch.cuda.synchronize()
        want = full.cpu().numpy()[povs[:, 0], povs[:, 1]]
        assert np.array_equal(got.cpu().numpy(), want)


@pytest.mark.parametrize("rows,cols,n,rng,h0", [(90, 70, 180, 0.0, 1.5), (60, 130, 24, 700.0, 8.0),
                                                (33, 64, 4, 320.0, 2.0), (2, 65, 1, 0.0, 1.5)])
def test_direct_points_match_the_oracle_definition(ctx, ctx32, orc, rows, cols, n, rng, h0):
    import torch
    dem = terrain.fractal_dem(rows, cols, 0.75, 500.0, seed=rows * cols)
    d = torch.from_numpy(dem).cuda()
    povs = _povs(rows, cols, 30, seed=rows)
    cells = povs[:, 0].astype(np.int64) * cols + povs[:, 1]
    got = ctx.viewshed_points(d, 10.0, h0, n, rng, povs, mode="direct").cpu().numpy()
    o64 = orc.direct_viewshed(dem, 10.0, h0, n, rng, prec=64, cells=cells)
    np.testing.assert_allclose(got, o64, rtol=FP32_RTOL, atol=0)
    got32 = ctx32.viewshed_points(d, 10.0, h0, n, rng, povs, mode="direct").cpu().numpy()
    o32 = orc.direct_viewshed(dem, 10.0, h0, n, rng, prec=32, cells=cells)
    np.testing.assert_allclose(got32, o32, rtol=FP32_RTOL, atol=0)


def test_direct_equals_sdem_when_lines_hit_cell_centres(ctx):
    import torch
    dem = terrain.fractal_dem(80, 95, 0.8, 400.0, seed=3)
    d = torch.from_numpy(dem).cuda()
    povs = _povs(80, 95, 50, seed=4)
    for n in (1, 2, 4):
        a = ctx.viewshed_points(d, 10.0, 1.5, n, 0.0, povs, mode="sdem").cpu().numpy()
        b = ctx.viewshed_points(d, 10.0, 1.5, n, 0.0, povs, mode="direct").cpu().numpy()
        assert np.array_equal(a, b)


def test_multiple_viewshed_of_ten_povs_at_paper_scale(ctx):
    """The paper's first experiment: the viewsheds of 10 random POVs of the
    2000 x 2000 DEM; each equals the total viewshed map's value."""
    import torch
    w = terrain.WORKLOADS["tvs2000"]
    dem = terrain.workload_dem("tvs2000")
    d = torch.from_numpy(dem).cuda()
    povs = _povs(2000, 2000, 10, seed=2003)[:10]
    got = ctx.viewshed_points(d, w["step"], w["h0"], w["n"], 0.0, povs).cpu().numpy()
    full = ctx.total_viewshed_device(d, w["step"], w["h0"], w["n"], 0.0).cpu().numpy()
    assert np.array_equal(got, full[povs[:, 0], povs[:, 1]])
    direct = ctx.viewshed_points(d, w["step"], w["h0"], w["n"], 0.0, povs, mode="direct").cpu().numpy()
    assert np.all(np.isfinite(direct)) and np.all(direct > 0)


def test_points_refuse_bad_arguments(ctx):
    import torch
    d = torch.zeros((10, 12), device="cuda")
    with pytest.raises(tvs.TvsError) as ei:
        ctx.viewshed_points(d, 10.0, 1.5, 8, 0.0, [[10, 0]])
    assert ei.value.code == TVS_ERR_ARG and "outside" in str(ei.value)
    with pytest.raises(tvs.TvsError):
        ctx.viewshed_points(d, 10.0, 1.5, 8, 0.0, np.zeros((0, 2)))


def _ambiguous(rows, cols, n, povs, eps=1e-9):
    """Cells within eps of a sector boundary for some POV (numpy's and the
    device's double atan2 may round those either way)."""
    ii, jj = np.mgrid[0:rows, 0:cols]
    amb = np.zeros((rows, cols), bool)
    for (i0, j0) in povs:
        q = np.arctan2((ii - i0).astype(np.float64), (jj - j0).astype(np.float64)) * n / np.pi
        f = q - np.floor(q)
        amb |= (np.abs(f - 0.5) < eps) & ~((ii == i0) & (jj == j0))
    return amb


@pytest.mark.parametrize("rows,cols,n,rng,h0,npov", [(120, 90, 180, 0.0, 1.5, 3), (64, 200, 36, 900.0, 10.0, 5),
                                                     (2000, 2000, 180, 0.0, 1.5, 2), (33, 64, 4, 320.0, 2.0, 4),
                                                     (150, 170, 1000, 0.0, 5.0, 3), (41, 37, 12, 0.0, 1.5, 6),
                                                     (3, 16384, 4, 0.0, 1.5, 3)])
def test_visibility_map_matches_the_oracle(ctx, ctx32, orc, rows, cols, n, rng, h0, npov):
    import torch
    dem = terrain.fractal_dem(rows, cols, 0.8, 900.0 if rows < 1000 else 1500.0, seed=rows + n)
    d = torch.from_numpy(dem).cuda()
    povs = _povs(rows, cols, npov, seed=rows + 1)[:npov]
    amb = _ambiguous(rows, cols, n, povs)
    assert amb.mean() < 1e-3
    for c, prec in ((ctx, 64), (ctx32, 32)):
        got = c.visibility_map(d, 10.0, h0, n, rng, povs).cpu().numpy()
        want = orc.visibility_map(dem, 10.0, h0, n, rng, prec=prec, povs=povs)
        assert np.array_equal(got[~amb], want[~amb]), prec
        assert got.max() <= npov and all(got[p[0], p[1]] >= 1 for p in povs)


def test_visibility_map_refuses_bad_arguments(ctx):
    import torch
    d = torch.zeros((10, 12), device="cuda")
    with pytest.raises(tvs.TvsError) as ei:
        ctx.visibility_map(d, 10.0, 1.5, 8, 0.0, [[0, 12]])
    assert ei.value.code == TVS_ERR_ARG


def test_profiling_counts_point_and_map_work(ctx):
    import torch
    dem = terrain.fractal_dem(70, 90, 0.8, 500.0, seed=12)
    d = torch.from_numpy(dem).cuda()
    povs = _povs(70, 90, 7, seed=12)
    ctx.profile(True)
    ctx.viewshed_points(d, 10.0, 1.5, 24, 400.0, povs, mode="sdem")
    ctx.visibility_map(d, 10.0, 1.5, 24, 400.0, povs)
    st = ctx.profile_read()
    ctx.profile(False)
    assert st["points"]["launches"] == 1 and st["points"]["total_ms"] > 0
    assert st["points"]["units"] == tvs.count_point_evals(70, 90, 24, povs, 10.0, 400.0, "sdem")
    assert st["map_flags"]["units"] == tvs.count_point_evals(70, 90, 24, povs, 10.0, 400.0, "direct")
    assert st["map_raster"]["units"] == 70 * 90 * len(povs)

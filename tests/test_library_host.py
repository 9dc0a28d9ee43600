"""CPU-only checks of the C-ABI library: it builds, loads, exports every
function include/tvs.h declares, and its host-side logic (direction table,
work count, argument checks) agrees with the oracle.  No GPU compute here."""
import ctypes as C

import numpy as np
import pytest

import paper_2003_02200_gb300 as tvs


@pytest.fixture(scope="module")
def lib():
    return tvs.load()


def test_library_exports_every_declared_function(lib):
    names = tvs.declared_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name
    assert lib.tvs_abi_version() == 2


@pytest.mark.parametrize("n,rows,cols", [(180, 100, 100), (7, 13, 29), (360, 50, 21), (1, 2, 2), (4, 9, 5)])
def test_direction_table_matches_oracle(orc, n, rows, cols):
    for k in range(n):
        a = tvs.direction(n, k, rows, cols, 10.0, 1234.0)
        b = orc.direction(n, k, rows, cols, 10.0, 1234.0)
        for f in ("frame", "m", "H", "W", "t_fx", "D", "K"):
            assert a[f] == b[f], (k, f)
        assert a["g"] == b["g"] and a["t"] == b["t"]
        assert a["R"] == a["H"] + a["D"]


@pytest.mark.parametrize("rows,cols,n,step,rng", [
    (12, 15, 4, 10.0, 0.0), (23, 17, 9, 10.0, 0.0), (40, 40, 180, 10.0, 0.0), (31, 20, 16, 5.0, 42.0),
    (2, 2, 1, 1.0, 0.0), (50, 3, 8, 1.0, 3.0)])
def test_eval_count_matches_oracle(orc, rows, cols, n, step, rng):
    assert tvs.count_evals(rows, cols, n, step, rng) == orc.count_evals(rows, cols, n, step, rng)


def test_eval_count_paper_scale_closed_form():
    """For a square DEM with unlimited range every direction's work is about
    sum over rows of L^2; for 2000^2 and 180 directions about 0.85 W^3 n."""
    E = tvs.count_evals(2000, 2000, 180, 10.0, 0.0)
    assert 0.7 * 2000 ** 3 * 180 < E < 1.0 * 2000 ** 3 * 180


def test_host_argument_errors(lib):
    info = tvs._binding.DirectionInfo()
    assert lib.tvs_direction(0, 0, 10, 10, 1.0, 0.0, C.byref(info)) == tvs._binding.TVS_ERR_ARG
    assert lib.tvs_direction(8, 8, 10, 10, 1.0, 0.0, C.byref(info)) == tvs._binding.TVS_ERR_ARG
    assert lib.tvs_direction(8, 1, 1, 10, 1.0, 0.0, C.byref(info)) == tvs._binding.TVS_ERR_ARG
    assert lib.tvs_direction(8, 1, 10, 10, 0.0, 0.0, C.byref(info)) == tvs._binding.TVS_ERR_ARG
    assert lib.tvs_count_evals(1, 10, 4, 1.0, 0.0) < 0
    assert lib.tvs_count_evals(10, 10, 4, 1.0, float("nan")) < 0
    assert b"n_sectors" in lib.tvs_last_error(None) or lib.tvs_last_error(None)
    h = C.c_void_p()
    assert lib.tvs_create(None, 0, 0) == tvs._binding.TVS_ERR_ARG
    assert lib.tvs_total_viewshed(None, None, 4, 4, 1.0, 1.0, 4, 0.0, None) == tvs._binding.TVS_ERR_ARG
    lib.tvs_destroy(None)
    del h
    # request server: argument checks that need no GPU
    t = C.c_int64(0)
    assert lib.tvs_server_create(0, None, None) == tvs._binding.TVS_ERR_ARG
    bad = tvs._binding.ServerConfig(0, 0, 0.0, 0.0, 0, 7, 0, 0)          # unknown policy
    assert lib.tvs_server_create(0, C.byref(bad), C.byref(C.c_void_p())) == tvs._binding.TVS_ERR_ARG
    bad = tvs._binding.ServerConfig(0, 0, -1.0, 0.0, 0, 0, 0, 0)         # negative step size
    assert lib.tvs_server_create(0, C.byref(bad), C.byref(C.c_void_p())) == tvs._binding.TVS_ERR_ARG
    assert lib.tvs_server_submit(None, None, 4, 4, 1.0, 1.0, 4, 0.0, None, C.byref(t)) == tvs._binding.TVS_ERR_ARG
    assert lib.tvs_server_wait(None, 1, 0.0) == tvs._binding.TVS_ERR_ARG
    assert lib.tvs_server_query(None, 1, None) == tvs._binding.TVS_ERR_ARG
    assert lib.tvs_server_clock(None) == 0.0
    assert lib.tvs_server_forget(None, 1) == tvs._binding.TVS_ERR_ARG
    lib.tvs_server_destroy(None)


def test_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(tvs.TvsError) as ei:
        tvs.Context(0)
    assert ei.value.code == tvs._binding.TVS_ERR_CUDA
    with pytest.raises(tvs.TvsError) as ei:
        tvs.Server(0)
    assert ei.value.code == tvs._binding.TVS_ERR_CUDA


def test_terrain_generator_is_seeded_and_shaped():
    from paper_2003_02200_gb300 import terrain
    a = terrain.fractal_dem(64, 80, 0.8, 500.0, seed=1)
    b = terrain.fractal_dem(64, 80, 0.8, 500.0, seed=1)
    assert a.dtype == np.float32 and a.shape == (64, 80)
    assert np.array_equal(a, b)
    assert a.min() == 0.0 and abs(a.max() - 500.0) < 1e-3
    s = terrain.fractal_dem(64, 64, 0.7, 100.0, seed=2, spike_frac=0.05)
    base = terrain.fractal_dem(64, 64, 0.7, 100.0, seed=2)
    raised = np.count_nonzero(s - base > 1.0)
    assert raised == round(0.05 * 64 * 64)
    tiles = terrain.batch_tiles(8)
    assert all(256 <= t["rows"] <= 1500 for t in tiles)
    reqs = terrain.request_stream(20)
    assert all(reqs[i]["arrival"] < reqs[i + 1]["arrival"] for i in range(19))


def _walk_len(i, j0, dirn, H, W, t_fx, K, base, direct):
    """Targets of one half-line, walked one by one with exact integers: the
    sample at column j has row a = base + floor(y / 2^32) and fraction
    y mod 2^32, y = j t_fx (SDEM, base row at column 0) or (j - j0) t_fx
    (DIRECT, through the cell); it is usable iff 0 <= j < W, a >= 0 and
    a <= H - 1 when the fraction is 0, a + 1 <= H - 1 otherwise."""
    n = 0
    for dd in range(1, K + 1):
        j = j0 + dirn * dd
        if not 0 <= j < W:
            break
        y = (j - j0 if direct else j) * t_fx
        a, fr = base + (y >> 32), y & 0xFFFFFFFF
        if a < 0 or (a > H - 1 if fr == 0 else a + 1 > H - 1):
            break
        n = dd
    return n


@pytest.mark.parametrize("rows,cols,n,step,rng", [(13, 29, 7, 10.0, 0.0), (40, 23, 16, 10.0, 120.0),
                                                  (2, 9, 1, 1.0, 0.0), (17, 17, 180, 5.0, 0.0)])
def test_point_eval_count_matches_brute_walks(orc, rows, cols, n, step, rng):
    r = np.random.default_rng(rows * cols)
    povs = np.concatenate([np.stack([r.integers(0, rows, 12), r.integers(0, cols, 12)], 1),
                           [[0, 0], [rows - 1, cols - 1], [0, cols - 1], [rows - 1, 0]]]).astype(np.int32)
    for mode in ("sdem", "direct"):
        want = 0
        for k in range(n):
            d = orc.direction(n, k, rows, cols, step, rng)
            H, W, t_fx, frame = d["H"], d["W"], d["t_fx"], d["frame"]
            K = W if d["K"] < 0 or d["K"] > W else d["K"]
            for iD, jD in povs.tolist():
                i, j0 = [(iD, jD), (jD, iD), (jD, W - 1 - iD), (H - 1 - iD, jD)][frame]
                if mode == "direct":
                    want += sum(_walk_len(i, j0, s, H, W, t_fx, K, i, True) for s in (1, -1))
                    continue
                y0 = j0 * t_fx
                frac = (y0 & 0xFFFFFFFF) != 0
                for v, ok in ((0, not frac or i <= H - 2), (1, frac and i >= 1)):
                    if ok:
                        base = i - (y0 >> 32) - v
                        want += sum(_walk_len(i, j0, s, H, W, t_fx, K, base, False) for s in (1, -1))
        assert tvs.count_point_evals(rows, cols, n, povs, step, rng, mode) == want, mode


# ------------------------------------------------------ batch planner (host) --

SMEM_OPTIN = 232448   # opt-in shared memory per CTA (227 KiB) the sweep layouts are sized for


def job_blocks(ij):
    """Runs of consecutive instances of one job, as (job, start, end)."""
    runs, s = [], 0
    for i in range(1, len(ij) + 1):
        if i == len(ij) or ij[i] != ij[s]:
            runs.append((int(ij[s]), s, i))
            s = i
    return runs


def test_plan_covers_every_direction_once_largest_first():
    jobs = [(300, 300, 90, 10.0, 0.0), (2000, 2000, 36, 10.0, 0.0), (800, 650, 45, 5.0, 900.0),
            (500, 2000, 24, 10.0, 0.0), (64, 64, 7, 10.0, 0.0)]
    ij, ik, ic = tvs._binding.debug_plan(jobs, 16 << 30, 152, SMEM_OPTIN, 1, 0)
    assert sorted(zip(ij.tolist(), ik.tolist())) == [(j, k) for j, J in enumerate(jobs) for k in range(J[2])]
    assert ic[0] == 0 and np.all(np.diff(ic) >= 0)
    runs = job_blocks(ij)
    assert len(runs) == len(jobs)                       # each job's directions stay together
    for j, s, e in runs:
        assert np.array_equal(ik[s:e], np.arange(jobs[j][2]))   # in direction order
    sides = [max(jobs[j][0], jobs[j][1]) for j, _, _ in runs]
    assert sides == sorted(sides, reverse=True)          # largest DEM first


def test_plan_cuts_chunks_on_direction_groups():
    """A budget that holds some but not all directions of a 2000 x 2000 job:
    every chunk but the last ends on a multiple of 8 directions (the FP32
    group sums, and so the results, do not depend on the budget)."""
    ij, ik, ic = tvs._binding.debug_plan([(2000, 2000, 180, 10.0, 0.0)], 1 << 30, 152, SMEM_OPTIN, 1, 0)
    assert ic.max() >= 2
    starts = np.flatnonzero(np.diff(ic)) + 1
    assert np.all(ik[starts] % 8 == 0)
    assert np.array_equal(ik, np.arange(180))


def test_plan_separates_sweep_layouts_for_certified_decisions():
    """Certified launches size their shared memory for their longest rows, so
    a 2000-sample DEM (a row per pair of warps) and a 300-sample one (a row
    per warp) take separate chunks; FP32 decisions, or no layout information,
    let them share one."""
    jobs = [(300, 300, 180, 10.0, 0.0), (2000, 2000, 180, 10.0, 0.0), (280, 310, 90, 10.0, 0.0)]
    ij, _, ic = tvs._binding.debug_plan(jobs, 64 << 30, 152, SMEM_OPTIN, 1, 0)
    for c in np.unique(ic):
        sides = {max(jobs[j][0], jobs[j][1]) >= 1500 for j in ij[ic == c]}
        assert len(sides) == 1
    assert ic.max() == 1
    for fp32, smem in ((1, SMEM_OPTIN), (0, 0)):
        _, _, ic2 = tvs._binding.debug_plan(jobs, 64 << 30, 152, smem, 1, fp32)
        assert ic2.max() == 0


def test_plan_errors():
    with pytest.raises(tvs.TvsError):                    # one direction does not fit
        tvs._binding.debug_plan([(2000, 2000, 180, 10.0, 0.0)], 64 << 20, 152, SMEM_OPTIN)
    with pytest.raises(tvs.TvsError):                    # bad job
        tvs._binding.debug_plan([(1, 2000, 180, 10.0, 0.0)], 1 << 30, 152, SMEM_OPTIN)
    lib = tvs.load()
    one = np.array([100], np.int32)
    n = np.array([16], np.int32)
    d = np.array([10.0])
    z = np.array([0.0])
    out = np.zeros(16, np.int32)
    cnt = C.c_int32(0)
    rc = lib.tvs_debug_plan(one.ctypes.data, one.ctypes.data, n.ctypes.data, d.ctypes.data, z.ctypes.data, 1,
                            1 << 30, 152, 0, 1, 0, out.ctypes.data, out.ctypes.data, out.ctypes.data, 15,
                            C.byref(cnt), C.byref(cnt))
    assert rc == tvs._binding.TVS_ERR_ARG               # inst_cap below the number of directions

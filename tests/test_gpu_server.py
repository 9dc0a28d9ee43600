"""Request server (continuous batching): each result is the same alone and in
the mix, late arrivals share steps with running requests, admission waits for
room in the HBM arena, and bad requests are refused."""
import time

import numpy as np
import pytest

import paper_2003_02200_gb300 as tvs
from paper_2003_02200_gb300 import terrain
from paper_2003_02200_gb300._binding import TVS_ERR_ARG, TVS_ERR_OOM

pytestmark = pytest.mark.gpu

# (rows, cols, directions, step m, observer m, max range m): uneven shapes,
# degenerate strips, every frame, limited and unlimited range
REQS = [(40, 60, 36, 10.0, 1.5, 0.0), (130, 97, 45, 5.0, 12.0, 0.0), (64, 64, 180, 30.0, 2.0, 600.0),
        (300, 210, 90, 10.0, 1.5, 0.0), (2, 500, 8, 10.0, 3.0, 0.0), (257, 3, 16, 10.0, 1.0, 0.0),
        (90, 90, 90, 10.0, 25.0, 900.0), (517, 433, 180, 10.0, 1.5, 5000.0)]
BIG = 7
SLOT = 128 << 20


def _dems(seed):
    return [terrain.fractal_dem(r, c, 0.6 + 0.05 * (i % 5), 300.0 + 100.0 * i, seed + i)
            for i, (r, c, *_) in enumerate(REQS)]


@pytest.fixture(scope="module")
def alone():
    """Every request computed on its own through the single-DEM host API."""
    dems = _dems(500)
    with tvs.Context(0) as ctx:
        outs = [ctx.total_viewshed(d, s, h, n, rg) for d, (_, _, n, s, h, rg) in zip(dems, REQS)]
    return dems, outs


def _submit_all(srv, dems, order=None):
    order = range(len(REQS)) if order is None else order
    return {i: srv.submit(dems[i], REQS[i][3], REQS[i][4], REQS[i][2], REQS[i][5]) for i in order}


@pytest.mark.parametrize("policy", ["deadline", "fifo", "srpt"])
def test_results_are_the_same_alone_and_in_the_mix(alone, policy):
    dems, want = alone
    # small steps: requests are sliced over several steps, each shared with others
    with tvs.Server(0, hbm_budget_bytes=2 * SLOT + (64 << 20), step_slot_bytes=SLOT, step_evals=3e8,
                    policy=policy) as srv:
        tickets = _submit_all(srv, dems)
        outs = {i: srv.wait(t, timeout=300) for i, t in tickets.items()}
        infos = {i: srv.query(t) for i, t in tickets.items()}
        st = srv.stats()
    for i in range(len(REQS)):
        np.testing.assert_array_equal(outs[i], want[i])
    assert all(q["state_name"] == "done" and q["error"] == 0 for q in infos.values())
    assert st["completed"] == len(REQS) and st["failed"] == 0 and st["queued"] == 0 and st["active"] == 0
    assert st["max_step_jobs"] >= 2                       # requests shared steps
    assert infos[BIG]["steps"] >= 2                       # and were sliced over several
    evals = [tvs.count_evals(r, c, n, s, rg) for (r, c, n, s, _, rg) in REQS]
    assert [q["evals"] for q in infos.values()] == evals
    assert st["evals"] == sum(evals)
    for q in infos.values():
        assert 0.0 <= q["t_submit"] <= q["t_admit"] <= q["t_first"] <= q["t_done"]


# FP32 blend and FP32 group sums of 8 directions against the FP64 sums
FP32_RTOL = 4e-6


def test_served_results_match_the_fp64_oracle(alone, orc):
    """Every served result against the oracle itself (FP64 definition):
    certified decisions make each per-sample measure the definition's, so a
    served area differs from the oracle's only by single-precision sums --
    every cell of the small requests, 400 sampled cells of the largest."""
    dems, _ = alone
    with tvs.Server(0, hbm_budget_bytes=2 * SLOT + (64 << 20), step_slot_bytes=SLOT, step_evals=3e8,
                    policy="deadline") as srv:
        tickets = _submit_all(srv, dems)
        outs = {i: srv.wait(t, timeout=300) for i, t in tickets.items()}
    for i, (r, c, n, step, h0, rng) in enumerate(REQS):
        if r * c <= 40000:
            want = orc.total_viewshed(dems[i], step, h0, n, rng, prec=64)
            np.testing.assert_allclose(outs[i], want, rtol=FP32_RTOL, atol=0, err_msg=f"request {i}")
        else:
            cells = np.random.default_rng(i).choice(r * c, size=400, replace=False)
            want = orc.total_viewshed(dems[i], step, h0, n, rng, prec=64, cells=cells)
            np.testing.assert_allclose(outs[i].ravel()[cells], want, rtol=FP32_RTOL, atol=0,
                                       err_msg=f"request {i}")


def test_late_arrivals_join_and_finish_first(alone):
    """Small requests submitted while a large one runs join its next steps and,
    under the deadline policy, finish before it."""
    dems, want = alone
    with tvs.Server(0, hbm_budget_bytes=2 * SLOT + (64 << 20), step_slot_bytes=SLOT, step_evals=2e8) as srv:
        big = srv.submit(dems[BIG], REQS[BIG][3], REQS[BIG][4], REQS[BIG][2], REQS[BIG][5])
        while srv.query(big)["state_name"] != "running":
            time.sleep(1e-4)
        small = _submit_all(srv, dems, order=[0, 2, 4, 5])
        got = {i: srv.wait(t, timeout=300) for i, t in small.items()}
        got[BIG] = srv.wait(big, timeout=300)
        qb = srv.query(big)
        qs = [srv.query(t) for t in small.values()]
    for i, o in got.items():
        np.testing.assert_array_equal(o, want[i])
    assert qb["steps"] >= 2
    assert all(q["t_first"] > qb["t_first"] and q["t_done"] < qb["t_done"] for q in qs)


def test_admission_waits_for_arena_room(alone):
    """An arena smaller than the whole mix: the large request, submitted last,
    is admitted only once earlier requests have finished and left room."""
    dems, want = alone
    cells = [r * c for (r, c, *_) in REQS]
    need_big = 24 * cells[BIG]
    arena = need_big + 24 * max(cells[:BIG]) // 2
    with tvs.Server(0, hbm_budget_bytes=2 * SLOT + arena, step_slot_bytes=SLOT, step_evals=3e8) as srv:
        tickets = _submit_all(srv, dems)
        outs = {i: srv.wait(t, timeout=300) for i, t in tickets.items()}
        infos = {i: srv.query(t) for i, t in tickets.items()}
        st = srv.stats()
    for i in range(len(REQS)):
        np.testing.assert_array_equal(outs[i], want[i])
    assert st["arena_bytes"] == arena
    assert st["arena_peak_bytes"] <= st["arena_bytes"]
    assert infos[BIG]["t_admit"] >= min(q["t_done"] for i, q in infos.items() if i != BIG)


def test_max_active_limits_admission(alone):
    dems, want = alone
    with tvs.Server(0, hbm_budget_bytes=2 * SLOT + (64 << 20), step_slot_bytes=SLOT, step_evals=3e8,
                    max_active=1, lanes=1) as srv:
        tickets = _submit_all(srv, dems, order=[0, 1, 2, 4])
        outs = {i: srv.wait(t, timeout=300) for i, t in tickets.items()}
        infos = [srv.query(t) for t in tickets.values()]
        st = srv.stats()
    for i, o in outs.items():
        np.testing.assert_array_equal(o, want[i])
    assert st["max_step_jobs"] == 1
    for a, b in zip(infos, infos[1:]):
        assert b["t_admit"] >= a["t_done"]


def test_server_refuses_bad_requests_and_configs():
    with pytest.raises(tvs.TvsError) as ei:
        tvs.Server(0, lanes=3)
    assert ei.value.code == TVS_ERR_ARG
    with tvs.Server(0, hbm_budget_bytes=2 * SLOT + (4 << 20), step_slot_bytes=SLOT) as srv:
        dem = terrain.fractal_dem(10, 12, 0.8, 100.0, seed=1)
        for args in [(0.0, 1.5), (10.0, float("nan"))]:
            with pytest.raises(tvs.TvsError) as ei:
                srv.submit(dem, *args)
            assert ei.value.code == TVS_ERR_ARG
        bad = dem.copy()
        bad[3, 4] = np.inf
        with pytest.raises(tvs.TvsError) as ei:
            srv.submit(bad, 10.0, 1.5)
        assert ei.value.code == TVS_ERR_ARG
        with pytest.raises(tvs.TvsError) as ei:                 # 24 MB of residents > 4 MiB arena
            srv.submit(np.zeros((1000, 1000), np.float32), 10.0, 1.5)
        assert ei.value.code == TVS_ERR_OOM
        with pytest.raises(tvs.TvsError) as ei:
            srv.query(987654)
        assert ei.value.code == TVS_ERR_ARG
        t = srv.submit(dem, 10.0, 1.5, 24)
        assert srv.wait(t, timeout=60).shape == dem.shape
        assert srv.stats()["completed"] == 1
        srv.forget(t)
        with pytest.raises(tvs.TvsError) as ei:        # the record is gone
            srv.query(t)
        assert ei.value.code == TVS_ERR_ARG


def test_close_with_requests_in_flight_finishes_admitted_ones():
    dems = _dems(700)
    srv = tvs.Server(0, hbm_budget_bytes=2 * SLOT + (64 << 20), step_slot_bytes=SLOT, step_evals=3e8)
    for i in range(len(REQS)):
        srv.submit(dems[i], REQS[i][3], REQS[i][4], REQS[i][2], REQS[i][5])
    t0 = time.time()
    srv.close()
    assert time.time() - t0 < 120


def test_a_failed_step_fails_unfinished_requests_and_refuses_new_ones():
    """Host-side failure injection (no GPU fault): enqueueing the third step
    fails as a CUDA error would; every unfinished request fails with the
    error, requests finished before stay done, new submissions are refused,
    and shutdown does not hang."""
    from paper_2003_02200_gb300._binding import TVS_ERR_CUDA, TVS_ERR_STATE
    dems = _dems(900)
    srv = tvs.Server(0, hbm_budget_bytes=2 * SLOT + (64 << 20), step_slot_bytes=SLOT, step_evals=2e8,
                     policy="fifo", fail_after_steps=2)
    # the large request first: it needs far more than two steps; the others may
    # be refused already if the failure has happened by the time they arrive
    tickets = []
    for i in (BIG, 0, 1, 2):
        try:
            tickets.append(srv.submit(dems[i], REQS[i][3], REQS[i][4], REQS[i][2], REQS[i][5]))
        except tvs.TvsError as e:
            assert e.code == TVS_ERR_STATE and "injected" in str(e)
    codes = []
    for t in tickets:
        try:
            srv.wait(t, timeout=120)
            codes.append(0)
        except tvs.TvsError as e:
            codes.append(e.code)
            assert "injected" in str(e)
    assert codes[0] == TVS_ERR_CUDA                 # the large request cannot finish in two steps
    assert all(c in (0, TVS_ERR_CUDA) for c in codes)
    infos = [srv.query(t) for t in tickets]
    assert all(q["state_name"] in ("done", "failed") for q in infos)
    assert srv.stats()["failed"] >= 1
    with pytest.raises(tvs.TvsError) as ei:
        srv.submit(dems[0], 10.0, 1.5, 8)
    assert ei.value.code == TVS_ERR_STATE
    t0 = time.time()
    srv.close()
    assert time.time() - t0 < 60

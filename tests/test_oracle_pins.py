"""Pins of the oracle against what the paper and the mathematics fix (CPU only).

Each test names the passage it checks.  None of them re-types the oracle's
code: the brute force in ``refgeom`` builds explicit interval lists from
floating-point geometry, and the other tests use closed forms, invariants and
a hand-derived example.
"""
import math
import os

import numpy as np
import pytest

import refgeom

pytestmark = pytest.mark.filterwarnings("ignore")

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rand_dem(rows, cols, seed, scale=20.0, offset=0.0):
    rng = np.random.default_rng(seed)
    return (offset + rng.random((rows, cols)) * scale).astype(np.float32)


def scale_of(n, step):
    return math.pi / (2 * n) * step * step


def exact_rtol(n):
    """Tolerance of a closed form: 1e-12 when every direction has t in {0, 1}
    (no interpolation); otherwise 1e-9, the gap between the oracle's 32.32
    fixed-point tangent and the test's floating-point one (|dt| <= 2^-33)."""
    return 1e-12 if n in (1, 2, 4) else 1e-9


# --- brute force on small grids (Alg. 1-4, 6, 8, 9) -------------------------

@pytest.mark.parametrize("rows,cols,n,max_range", [
    (16, 16, 1, 0.0), (16, 16, 2, 0.0), (12, 16, 4, 0.0), (16, 12, 8, 0.0), (9, 13, 16, 0.0),
    (7, 6, 180, 0.0), (11, 9, 7, 0.0), (16, 16, 8, 55.0), (10, 14, 180, 42.0), (2, 9, 5, 0.0),
    (9, 2, 12, 0.0),
])
@pytest.mark.parametrize("prec", [64, 32])
def test_brute_force_small_grids(orc, rows, cols, n, max_range, prec):
    dem = rand_dem(rows, cols, seed=rows * 100 + cols * 7 + n)
    step, h0 = 10.0, 1.5
    want = refgeom.brute_total_viewshed(dem, step, h0, n, max_range)
    got = orc.total_viewshed(dem, step, h0, n, max_range, prec=prec).reshape(-1)
    np.testing.assert_allclose(got, want, rtol=1e-9, atol=0)


@pytest.mark.parametrize("n", [5, 180])
def test_brute_force_16x16_sampled_cells(orc, n):
    dem = rand_dem(16, 16, seed=77 + n)
    cells = np.random.default_rng(5).choice(256, size=12, replace=False)
    want = refgeom.brute_total_viewshed(dem, 5.0, 2.0, n, 0.0, cells=cells)
    got = orc.total_viewshed(dem, 5.0, 2.0, n, 0.0, cells=cells)
    np.testing.assert_allclose(got, want, rtol=1e-9, atol=0)


@pytest.mark.parametrize("n", [3, 8, 180])
def test_brute_force_per_half_line_cv_exact(orc, n):
    """Every virtual POV's forward and backward cv is the same integer."""
    dem = rand_dem(9, 12, seed=n)
    rng = np.random.default_rng(n)
    for _ in range(40):
        i, j, k = int(rng.integers(9)), int(rng.integers(12)), int(rng.integers(n))
        want = refgeom.cell_direction_cv(dem, 10.0, 1.5, n, 0.0, i, j, k)
        got = orc.cell_direction(dem, 10.0, 1.5, n, 0.0, 64, i, j, k)
        assert len(got) == len(want)
        for g, w in zip(got, want):
            assert (g["cv_fwd"], g["cv_bwd"]) == (w["cv_fwd"], w["cv_bwd"])
            assert g["w"] == pytest.approx(w["w"], abs=1e-9)


# --- flat terrain: closed forms (section 3.1 ring-sector area) ---------------

def flat_expected(rows, cols, n, step, max_range, fn):
    """(pi/(2n)) step^2 sum_k g_k sum_v w_v (fn(L_fwd) + fn(L_bwd))."""
    out = np.zeros((rows, cols))
    for i in range(rows):
        for j in range(cols):
            acc = 0.0
            for k in range(n):
                acc += sum(g * w * (fn(lf) + fn(lb))
                           for w, lf, lb, g in refgeom.walk_lengths(rows, cols, n, step, max_range, i, j, k))
            out[i, j] = scale_of(n, step) * acc
    return out


@pytest.mark.parametrize("rows,cols,n,max_range", [
    (13, 17, 1, 0.0), (13, 17, 2, 0.0), (13, 17, 4, 0.0), (11, 9, 8, 0.0), (7, 8, 180, 0.0),
    (12, 12, 6, 35.0),
])
@pytest.mark.parametrize("prec", [64, 32])
def test_flat_everything_visible(orc, rows, cols, n, max_range, prec):
    """h0 > 0 on flat ground: slopes -h0/dd strictly increase, every target is
    visible and each half-line's measure is L^2 (one segment [0, L))."""
    dem = np.full((rows, cols), 321.25, np.float32)
    got = orc.total_viewshed(dem, 10.0, 1.5, n, max_range, prec=prec)
    want = flat_expected(rows, cols, n, 10.0, max_range, lambda L: L * L)
    np.testing.assert_allclose(got, want, rtol=exact_rtol(n), atol=0)


@pytest.mark.parametrize("n", [4, 7, 180])
def test_flat_zero_observer_height_ties(orc, n):
    """0 m terrain with h0 = 0: every slope is 0, the strict test of Alg. 3/8
    hides every target after the first, so a half-line measures 4 when it
    has at least two targets (segment [0,2)), 1 with one target, 0 with none.
    It also checks that real 0 m elevations are not dropped (nzSet reading)."""
    rows, cols = 8, 9
    dem = np.zeros((rows, cols), np.float32)
    got = orc.total_viewshed(dem, 1.0, 0.0, n)
    want = flat_expected(rows, cols, n, 1.0, 0.0, lambda L: 4 if L >= 2 else L)
    np.testing.assert_allclose(got, want, rtol=exact_rtol(n), atol=0)


def test_flat_large_n_approaches_rectangle_area(orc):
    """With many directions the summed ring sectors of a flat DEM fill the
    rectangle spanned by the cell centres (Pappus / ring-sector area), up to the
    one-step discretisation at the far edge."""
    rows = cols = 61
    dem = np.zeros((rows, cols), np.float32)
    cells = [30 * cols + 30, 0, 5 * cols + 40]
    got = orc.total_viewshed(dem, 1.0, 1.5, 180, cells=cells)
    area = (rows - 1) * (cols - 1)
    for v in got:
        assert abs(v - area) / area < 0.05


# --- single wall and single cone: analytic shadows -------------------------

def half_lines_n4(rows, cols, i, j):
    """For n = 4 (t in {0, 1}, no interpolation): per direction, the cells of
    both half-lines from (i, j) in DEM coordinates, nearest first, and g."""
    dirs = [((0, 1), 1.0), ((1, 1), 2.0), ((1, 0), 1.0), ((1, -1), 2.0)]
    res = []
    for (di, dj), g in dirs:
        lines = []
        for sgn in (1, -1):
            cells = []
            s = 1
            while 0 <= i + sgn * s * di < rows and 0 <= j + sgn * s * dj < cols:
                cells.append((i + sgn * s * di, j + sgn * s * dj))
                s += 1
            lines.append(cells)
        res.append((lines, g))
    return res


def test_single_wall_shadow(orc):
    """One DEM column raised to a wall above the observer: a POV on flat
    ground sees up to and including the wall cell at distance a, and nothing
    behind it, so that half-line measures (a+1)^2 (or L^2 if the wall is the
    last target).  Every other half-line is flat: L^2."""
    rows, cols, c, Hw, h0 = 9, 11, 6, 50.0, 1.5
    dem = np.zeros((rows, cols), np.float32)
    dem[:, c] = Hw
    got = orc.total_viewshed(dem, 2.0, h0, 4)
    for i in range(rows):
        for j in range(cols):
            acc = 0.0
            for lines, g in half_lines_n4(rows, cols, i, j):
                for cells in lines:
                    L = len(cells)
                    hit = [s + 1 for s, (_, jj) in enumerate(cells) if jj == c]
                    if j != c and hit and hit[0] < L:
                        acc += g * (hit[0] + 1) ** 2
                    else:
                        acc += g * L * L
            assert got[i, j] == pytest.approx(scale_of(4, 2.0) * acc, rel=1e-12)


def cone_dem(rows, cols, cy, cx, Hc, R):
    ii, jj = np.mgrid[0:rows, 0:cols]
    rho = np.sqrt((ii - cy) ** 2 + (jj - cx) ** 2)
    return np.maximum(0.0, Hc * (1.0 - rho / R)).astype(np.float32)


def test_cone_shadow_along_axis(orc):
    """Observers on the apex row (n = 2, direction 0 runs along rows): toward
    the cone the profile is flat then linearly rising (convex, slopes strictly
    increase) up to the apex, then falls away below the sight line to the
    apex, so that half-line measures (a+1)^2 with a the distance to the apex;
    the other half-line is flat (L^2)."""
    rows, cols, cy, cx, Hc, R, h0 = 7, 31, 3, 15, 100.0, 6.0, 1.5
    dem = cone_dem(rows, cols, cy, cx, Hc, R)
    for j in list(range(0, cols)):
        if j == cx:
            continue
        res = orc.cell_direction(dem, 1.0, h0, 2, 0.0, 64, cy, j, 0)
        assert len(res) == 1 and res[0]["w"] == 1.0
        a = abs(j - cx)
        L_away = (cols - 1 - j) if j > cx else j
        L_to = j if j > cx else cols - 1 - j
        assert L_to > a
        got = res[0]["cv_fwd"] + res[0]["cv_bwd"]
        assert got == (a + 1) ** 2 + L_away ** 2, (j, got)


@pytest.mark.parametrize("n", [2, 4])
def test_cone_apex_sees_everything(orc, n):
    """From the apex of a convex cone every profile falls linearly then runs
    flat, slopes strictly increase, and the apex's value equals flat ground."""
    rows, cols, cy, cx = 15, 17, 7, 8
    dem = cone_dem(rows, cols, cy, cx, 80.0, 5.0)
    got = orc.total_viewshed(dem, 3.0, 1.5, n, cells=[cy * cols + cx])[0]
    acc = 0.0
    for k in range(n):
        acc += sum(g * w * (lf * lf + lb * lb)
                   for w, lf, lb, g in refgeom.walk_lengths(rows, cols, n, 3.0, 0.0, cy, cx, k))
    assert got == pytest.approx(scale_of(n, 3.0) * acc, rel=exact_rtol(n))


# --- invariants ---------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 4])
@pytest.mark.parametrize("prec", [64, 32])
def test_rotation_180_exact_for_axis_and_diagonal_directions(orc, n, prec):
    """Reversing both axes maps every line of direction k onto a line of the
    same direction with forward and backward swapped; with t in {0, 1} no
    interpolation is involved, so the map rotates exactly."""
    dem = rand_dem(9, 11, seed=3)
    a = orc.total_viewshed(dem, 10.0, 1.5, n, prec=prec)
    b = orc.total_viewshed(np.ascontiguousarray(dem[::-1, ::-1]), 10.0, 1.5, n, prec=prec)
    assert np.array_equal(a, b[::-1, ::-1])


def test_rotation_180_general_n_reported(orc):
    """For general n the sampled lines of the rotated DEM are not the rotated
    lines, so equality holds only up to interpolation; bounded loosely."""
    dem = rand_dem(12, 12, seed=4, scale=5.0)
    a = orc.total_viewshed(dem, 10.0, 1.5, 16)
    b = orc.total_viewshed(np.ascontiguousarray(dem[::-1, ::-1]), 10.0, 1.5, 16)[::-1, ::-1]
    rel = np.abs(a - b) / np.abs(a)
    assert np.median(rel) < 0.2


@pytest.mark.parametrize("prec", [64, 32])
def test_scale_invariance(orc, prec):
    """Doubling every elevation and h0 doubles every slope exactly (binary
    floating point), so every visibility decision and the output are
    bit-identical; doubling the step multiplies the area by exactly 4."""
    dem = rand_dem(10, 13, seed=9, scale=300.0)
    base = orc.total_viewshed(dem, 10.0, 1.5, 23, prec=prec)
    tall = orc.total_viewshed(dem * np.float32(2), 10.0, 3.0, 23, prec=prec)
    assert np.array_equal(base, tall)
    wide = orc.total_viewshed(dem, 20.0, 1.5, 23, prec=prec)
    assert np.array_equal(wide, 4.0 * base)


def _textbook_cv(profile, h):
    """Visible targets are those whose slope strictly exceeds the running
    maximum of the earlier slopes (prefix maximum); the measure follows from
    the branch-free form sum_d (v_{d-1} - v_d) d^2 + v_L L^2 with v_0 = 1."""
    L = len(profile)
    if L == 0:
        return 0
    s = (np.asarray(profile, np.float64) - h) / np.arange(1, L + 1)
    pm = np.maximum.accumulate(s)
    v = np.ones(L + 1, dtype=np.int64)
    v[2:] = s[1:] > pm[:-1]
    d = np.arange(1, L + 1)
    return int(np.sum((v[:-1] - v[1:]) * d * d) + v[L] * L * L)


def test_one_dimensional_textbook_and_branch_free_identity(orc):
    """n = 1 on a 2-row DEM: each row is an independent terrain profile and
    the oracle's stateful walk (Alg. 8) must equal the prefix-maximum visible
    set measured by the branch-free identity."""
    rng = np.random.default_rng(11)
    for trial in range(6):
        W = int(rng.integers(2, 60))
        dem = (rng.random((2, W)) * 30).astype(np.float32)
        if trial == 0:
            dem[:] = np.round(dem)          # integer heights: exact slope ties
        h0 = float(rng.choice([0.0, 1.5, 7.0]))
        for b in range(2):
            got = orc.line_cv(dem, 1.0, h0, 1, 0.0, 64, 0, b)
            row = dem[b].astype(np.float64)
            for j in range(W):
                want = _textbook_cv(row[j + 1:], row[j] + h0) + _textbook_cv(row[:j][::-1], row[j] + h0)
                assert got[j] == want


def test_golden_hand_derived_profile(orc):
    """The hand-worked example of tests/golden/profile_1d.txt."""
    spec = {}
    with open(os.path.join(GOLDEN, "profile_1d.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                key, *vals = line.split()
                spec[key] = [float(v) for v in vals]
    prof = np.array(spec["profile"], np.float32)
    dem = np.stack([prof, prof])
    h0 = spec["h0"][0]
    cv = np.array(spec["cv"])
    got = orc.total_viewshed(dem, 1.0, h0, 1)
    np.testing.assert_allclose(got[0], math.pi / 2 * cv, rtol=1e-15)
    np.testing.assert_allclose(got[1], math.pi / 2 * cv, rtol=1e-15)
    for prec in (64, 32):
        assert list(orc.line_cv(dem, 1.0, h0, 1, 0.0, prec, 0, 0)) == list(cv.astype(int))


def test_pappus_one_degree_sectors(orc):
    """With n = 180 each half-line sector is one degree wide, and a visible
    segment [r, R) adds (pi/360)(R^2 - r^2) (ring-sector area, section 3.1)."""
    rows, cols = 3, 40
    dem = np.zeros((rows, cols), np.float32)
    got = orc.total_viewshed(dem, 1.0, 1.5, 180, cells=[1 * cols + 0])[0]
    acc = 0.0
    for k in range(180):
        for w, lf, lb, g in refgeom.walk_lengths(rows, cols, 180, 1.0, 0.0, 1, 0, k):
            acc += w * ((lf * math.sqrt(g)) ** 2 + (lb * math.sqrt(g)) ** 2)
    assert got == pytest.approx(math.pi / 360 * acc, rel=exact_rtol(180))


# --- geometry, work count and argument checks --------------------------------

@pytest.mark.parametrize("n,rows,cols", [(180, 20, 31), (7, 13, 5), (4, 9, 9), (360, 17, 17)])
def test_line_ranges_match_float_geometry(orc, n, rows, cols):
    """Usable column range of every sampled line: the oracle's fixed-point
    range equals the float one (0 <= b + j t <= H-1)."""
    for k in range(n):
        d = orc.direction(n, k, rows, cols)
        frame, m = refgeom.frame_of(n, k)
        t = refgeom.tan_of(n, m)
        assert (d["frame"], d["m"]) == (frame, m)
        assert abs(d["t"] - t) < 1e-9
        for b in range(-d["D"] - 2, d["H"] + 2):
            js = [j for j in range(d["W"]) if 0.0 <= b + j * t <= d["H"] - 1]
            lo, hi = orc.line_range(n, k, rows, cols, b)
            if js:
                assert (lo, hi) == (js[0], js[-1])
                assert js == list(range(js[0], js[-1] + 1))
            else:
                assert hi < lo


def test_direction_frames_and_table(orc):
    """Directions k*pi/n (section 4.1: ns/2 relocations), four D4 frames,
    45 deg exactly t = 1, g = 1 + t^2 the (1/cos s)^2 factor of Alg. 7."""
    n = 180
    for k in range(n):
        d = orc.direction(n, k, 30, 40)
        theta = k * 180.0 / n
        alpha = d["m"] * 90.0 / n
        assert 0 <= alpha <= 45
        assert d["g"] == pytest.approx(1.0 / math.cos(math.radians(alpha)) ** 2, rel=1e-9)
        folded = {0: alpha, 1: 90 - alpha, 2: 90 + alpha, 3: 180 - alpha}[d["frame"]]
        assert folded == pytest.approx(theta, abs=1e-9)
        assert (d["H"], d["W"]) == ((30, 40) if d["frame"] in (0, 3) else (40, 30))
    assert orc.direction(n, 45, 30, 40)["t_fx"] == 1 << 32
    assert orc.direction(n, 135, 30, 40)["t_fx"] == 1 << 32
    assert orc.direction(n, 0, 30, 40)["t_fx"] == 0
    assert orc.direction(n, 90, 30, 40)["t_fx"] == 0


def test_eval_count_matches_visits_without_interpolation(orc):
    """Work count: with t in {0,1} every cell owns exactly one sampled POV, so
    the targets the oracle visits equal the counted evals."""
    dem = rand_dem(12, 15, seed=2)
    info = {}
    orc.total_viewshed(dem, 10.0, 1.5, 4, 0.0, info=info)
    assert info["evals_visited"] == orc.count_evals(12, 15, 4)
    info2 = {}
    orc.total_viewshed(dem, 10.0, 1.5, 4, 35.0, info=info2)
    assert info2["evals_visited"] == orc.count_evals(12, 15, 4, 10.0, 35.0)


def test_oracle_rejects_bad_arguments(orc):
    dem = rand_dem(4, 4, seed=1)
    with pytest.raises(ValueError):
        orc.total_viewshed(dem[:1], 10.0, 1.5, 4)
    with pytest.raises(ValueError):
        orc.total_viewshed(dem, 0.0, 1.5, 4)
    with pytest.raises(ValueError):
        orc.total_viewshed(dem, 10.0, 1.5, 0)
    bad = dem.copy()
    bad[1, 1] = np.nan
    with pytest.raises(ValueError):
        orc.total_viewshed(bad, 10.0, 1.5, 4)
    with pytest.raises(ValueError):
        orc.total_viewshed(dem, 10.0, float("inf"), 4)


# --- the singular viewshed by definition (Alg. 1-3), no virtual POVs ---------

@pytest.mark.parametrize("rows,cols,n,max_range", [
    (12, 12, 8, 0.0), (9, 14, 16, 0.0), (7, 6, 180, 0.0), (11, 9, 7, 0.0), (13, 10, 12, 47.0), (2, 9, 5, 0.0),
])
def test_direct_viewshed_brute_force(orc, rows, cols, n, max_range):
    """Alg. 1-3 with the line of sight through the POV cell itself: the oracle
    against explicit interval lists from floating-point geometry."""
    dem = rand_dem(rows, cols, seed=rows * 31 + cols + n)
    cells = list(range(rows * cols))
    got = orc.direct_viewshed(dem, 10.0, 1.5, n, max_range, prec=64, cells=cells)
    want = refgeom.brute_direct_viewshed(dem, 10.0, 1.5, n, max_range, cells=cells)
    np.testing.assert_allclose(got, want, rtol=1e-9, atol=0)


@pytest.mark.parametrize("n", [4, 9, 180])
def test_direct_viewshed_flat_closed_form(orc, n):
    """Flat ground and h0 > 0: every target is visible, so each half-line adds
    L^2 (L its number of targets), counted here with exact rational geometry:
    column j of the line through view cell (i, j0) is a target iff
    0 <= i + (j - j0) t <= H - 1 (Alg. 1-3 with the Alg. 6 sampling)."""
    from fractions import Fraction
    rows, cols = 14, 11
    dem = np.zeros((rows, cols), np.float32)
    cells = [0, 5, 3 * cols + 7, rows * cols - 1, 6 * cols + 5]
    got = orc.direct_viewshed(dem, 3.0, 2.0, n, 0.0, prec=64, cells=cells)
    for q, c in enumerate(cells):
        iD, jD = divmod(c, cols)
        acc = Fraction(0)
        for k in range(n):
            d = orc.direction(n, k, rows, cols)
            t = Fraction(d["t_fx"], 1 << 32)
            view = refgeom.View(dem, d["frame"])
            i, j0 = view.cell_to_view(iD, jD)
            for s in (1, -1):
                L = 0
                while 0 <= j0 + s * (L + 1) < view.W and 0 <= i + s * (L + 1) * t <= view.H - 1:
                    L += 1
                acc += (1 + t * t) * L * L
        want = scale_of(n, 3.0) * float(acc)
        assert got[q] == pytest.approx(want, rel=1e-12)


def test_direct_viewshed_zero_height_flat(orc):
    """Flat ground, h0 = 0: every slope is 0, so only the first target is
    strictly above the initial -inf maximum; a half-line with L >= 2 targets
    adds 2^2 (its segment closes at the second target), one with L = 1 adds 1."""
    rows, cols = 8, 8
    dem = np.zeros((rows, cols), np.float32)
    got = orc.direct_viewshed(dem, 1.0, 0.0, 1, 0.0, prec=64, cells=[3 * cols + 3, 0, cols - 1])
    # n = 1: the walk axis is the row; cell (3, 3) has 4 targets east and 3 west
    assert got[0] == pytest.approx(math.pi / 2 * (4 + 4), rel=1e-15)
    # (0, 0): 7 targets east, none west; (0, 7): none east, 7 west
    assert got[1] == pytest.approx(math.pi / 2 * 4, rel=1e-15)
    assert got[2] == pytest.approx(math.pi / 2 * 4, rel=1e-15)


@pytest.mark.parametrize("prec", [64, 32])
def test_direct_equals_sdem_when_lines_hit_cell_centres(orc, prec):
    """With n in {1, 2, 4} every direction has t in {0, 1}: the sampled lines of
    the skewed layout pass through every cell centre, so each cell is its own
    (single) virtual POV and sDEM and the definition coincide exactly."""
    dem = rand_dem(15, 12, seed=9)
    cells = list(range(15 * 12))
    for n in (1, 2, 4):
        a = orc.total_viewshed(dem, 10.0, 1.5, n, 0.0, prec=prec, cells=cells)
        b = orc.direct_viewshed(dem, 10.0, 1.5, n, 0.0, prec=prec, cells=cells)
        np.testing.assert_array_equal(a, b)


def test_direct_differs_from_sdem_only_by_discretisation(orc):
    """For general n the two differ (virtual POVs on whole-row lines against the
    cell's own lines) but stay close on smooth terrain: the sDEM discretisation
    error the paper reports against TVS (section 5) is of the order of 1 %."""
    rows, cols = 40, 40
    y, x = np.mgrid[0:rows, 0:cols]
    dem = (200.0 * np.sin(x / 9.0) * np.cos(y / 11.0)).astype(np.float32)
    cells = [c for c in range(rows * cols) if c % 7 == 0]
    a = orc.total_viewshed(dem, 10.0, 1.5, 60, 0.0, prec=64, cells=cells)
    b = orc.direct_viewshed(dem, 10.0, 1.5, 60, 0.0, prec=64, cells=cells)
    rel = np.abs(a - b) / b
    assert not np.array_equal(a, b)
    assert np.median(rel) < 0.05


# --- visibility map (which cells a POV sees; counts for several POVs) --------

def _ambiguous_cells(rows, cols, n, povs, eps=1e-9):
    amb = np.zeros((rows, cols), bool)
    for (i0, j0) in povs:
        for iD in range(rows):
            for jD in range(cols):
                if (iD, jD) != (i0, j0):
                    _, f = refgeom.sector_of(n, iD - i0, jD - j0)
                    amb[iD, jD] |= abs(f - 0.5) < eps
    return amb


@pytest.mark.parametrize("n,rows,cols,rng", [(8, 13, 17, 0.0), (36, 15, 12, 0.0), (7, 11, 11, 0.0),
                                              (20, 16, 14, 75.0)])
def test_visibility_map_brute_force(orc, n, rows, cols, rng):
    dem = rand_dem(rows, cols, seed=n + rows)
    povs = [(rows // 2, cols // 3), (0, cols - 1), (rows - 1, 2)]
    got = orc.visibility_map(dem, 10.0, 1.5, n, rng, prec=64, povs=povs)
    want = refgeom.brute_visibility_map(dem, 10.0, 1.5, n, povs, rng)
    amb = _ambiguous_cells(rows, cols, n, povs)
    assert np.array_equal(got[~amb], want[~amb])


@pytest.mark.parametrize("n", [4, 9, 36])
def test_visibility_map_flat_ground_reach(orc, n):
    """Flat ground, h0 > 0: every reached target is visible, so a cell is seen
    iff its sector's half-line through the POV still lies in the DEM at the
    cell's walk-axis column (exact rational geometry)."""
    from fractions import Fraction
    rows, cols = 12, 15
    dem = np.zeros((rows, cols), np.float32)
    i0, j0 = 5, 9
    got = orc.visibility_map(dem, 10.0, 2.0, n, 0.0, prec=64, povs=[(i0, j0)])
    amb = _ambiguous_cells(rows, cols, n, [(i0, j0)])
    for iD in range(rows):
        for jD in range(cols):
            if amb[iD, jD]:
                continue
            if (iD, jD) == (i0, j0):
                assert got[iD, jD] == 1
                continue
            kp, _ = refgeom.sector_of(n, iD - i0, jD - j0)
            d = orc.direction(n, kp % n, rows, cols)
            view = refgeom.View(dem, d["frame"])
            vi0, vj0 = view.cell_to_view(i0, j0)
            vi, vj = view.cell_to_view(iD, jD)
            plus = (d["frame"] <= 1) == (kp < n)
            dd = (vj - vj0) if plus else (vj0 - vj)
            t = Fraction(d["t_fx"], 1 << 32)
            reach = dd >= 1 and all(0 <= vi0 + (x if plus else -x) * t <= view.H - 1 for x in range(1, dd + 1))
            assert got[iD, jD] == int(reach), (iD, jD)


def test_visibility_map_counts_add_over_povs(orc):
    """The map of several POVs is the sum of their single maps (each cell
    counts the POVs that see it)."""
    dem = rand_dem(14, 13, seed=4)
    povs = [(1, 1), (7, 6), (13, 12), (3, 10)]
    together = orc.visibility_map(dem, 10.0, 1.5, 24, 0.0, prec=32, povs=povs)
    apart = sum(orc.visibility_map(dem, 10.0, 1.5, 24, 0.0, prec=32, povs=[p]) for p in povs)
    assert np.array_equal(together, apart)
    assert all(together[p] >= 1 for p in povs)


def _fp32_tie_cases():
    with open(os.path.join(GOLDEN, "fp32_ties.txt")) as f:
        lines = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]
    tfx = int(lines[0][1])
    cases, cur = [], None
    for ln in lines[1:]:
        if ln[0] == "case":
            cur = {"h0": float.fromhex(ln[2]), "rows": []}
            cases.append(cur)
        elif ln[0] == "row":
            cur["rows"].append([float.fromhex(v) for v in ln[1:]])
        elif ln[0] in ("cv32", "cv64"):
            cur[ln[0]] = [int(v) for v in ln[1:]]
    return tfx, cases


def test_golden_fp32_near_ties(orc):
    """tests/golden/fp32_ties.txt: near-tie lines of sight (direction 1 of 8,
    blended samples) whose measures were derived in exact rational arithmetic
    from the operation order of the FP32-decision reading ((1-r) a + r b,
    h = z + float(h0), (z - h) * rcp(d), all in single precision) and of the
    FP64 reading.  The generator kept cases that a
    division instead of rcp, a fused blend, h0 added unrounded, or the blend
    weight taken from the exact r would each change, so any of those mistakes
    in the oracle's FP32 mode fails here."""
    tfx, cases = _fp32_tie_cases()
    assert orc.direction(8, 1, 4, 8)["t_fx"] == tfx
    assert len(cases) >= 4
    for c in cases:
        dem = np.array(c["rows"], dtype=np.float32)
        assert np.array_equal(dem.astype(np.float64), np.array(c["rows"]))   # exact float32 values
        for prec in (32, 64):
            got = orc.line_cv(dem, 1.0, c["h0"], 8, 0.0, prec, 1, 0)
            assert got.tolist() == c[f"cv{prec}"], (prec, got.tolist(), c[f"cv{prec}"])
        assert c["cv32"] != c["cv64"]          # every case is a real FP32 / FP64 split

"""Test-side geometry and a brute-force viewshed, written independently of the
oracle's C code, used to pin the oracle.

Differences from the oracle on purpose:

* sample positions come from a floating-point tan(alpha) (no 32.32 fixed
  point), with the two rational cases (alpha = 0 and 45 deg) snapped to 0 and 1;
* a sampled line is the set of points Y(j) = b + j * t (b its integer row at
  j = 0), evaluated in floating point;
* visibility is found by rescanning all earlier slopes for every target, and
  the visible set is built as an explicit list of [start, end) intervals that
  is then measured (sum of end^2 - start^2), following Alg. 2 and Alg. 3.

The readings of the paper are the same as the oracle's (they are the
definition): directions theta_k = k*pi/n, the four D4 views chosen by integer
tests on k, the Kernel-1 blend (Alg. 6), the Kernel-3 weights (Alg. 9), strict
">" for visibility, segments closing at the first hidden target or at the last
target of the line, the Pappus factor pi/(2n) and step^2.
"""
from __future__ import annotations

import math

import numpy as np

AMBIGUOUS = 1e-9


def frame_of(n: int, k: int) -> tuple[int, int]:
    """(frame, m) with alpha = pi*m/(2n)."""
    if 4 * k < n:
        return 0, 2 * k
    if 4 * k < 2 * n:
        return 1, n - 2 * k
    if 4 * k < 3 * n:
        return 2, 2 * k - n
    return 3, 2 * n - 2 * k


def tan_of(n: int, m: int) -> float:
    if m == 0:
        return 0.0
    if 2 * m == n:          # alpha = pi/4
        return 1.0
    return math.tan(math.pi * m / (2 * n))


class View:
    """The D4 view of a DEM used by direction k (W is the walk axis)."""

    def __init__(self, dem: np.ndarray, frame: int):
        rows, cols = dem.shape
        self.frame = frame
        if frame == 0:
            self.V = dem
        elif frame == 1:
            self.V = dem.T
        elif frame == 2:
            self.V = dem.T[:, ::-1]
        else:
            self.V = dem[::-1, :]
        self.H, self.W = self.V.shape

    def cell_to_view(self, iD: int, jD: int) -> tuple[int, int]:
        rows = self.W if self.frame in (1, 2) else self.H
        if self.frame == 0:
            return iD, jD
        if self.frame == 1:
            return jD, iD
        if self.frame == 2:
            return jD, rows - 1 - iD
        return self.H - 1 - iD, jD


def _height(V: np.ndarray, Y: float, j: int) -> float:
    a = math.floor(Y)
    f = Y - a
    if f == 0.0:
        return float(V[a, j])
    return (1.0 - f) * float(V[a, j]) + f * float(V[a + 1, j])


def _usable(H: int, Y: float) -> bool:
    return 0.0 <= Y <= H - 1


def line_profile(view: View, t: float, j0: int, b: int, direction: int, K: int) -> list[float]:
    """Heights of the targets of the half-line of line b from column j0, nearest first."""
    out = []
    d = 1
    while d <= K:
        j = j0 + direction * d
        if j < 0 or j >= view.W:
            break
        Y = b + j * t
        if 0 < abs(Y - round(Y)) < AMBIGUOUS:
            raise AssertionError("sample too close to a grid line for a float reference")
        if not _usable(view.H, Y):
            break
        out.append(_height(view.V, Y, j))
        d += 1
    return out


def visible_intervals(h: float, profile: list[float]) -> list[tuple[int, int]]:
    """Visible [start, end) intervals of one half-line (Alg. 2 / Alg. 3)."""
    L = len(profile)
    slopes = [(profile[d - 1] - h) / d for d in range(1, L + 1)]
    visible = []
    for d in range(1, L + 1):
        earlier = slopes[: d - 1]
        visible.append(all(slopes[d - 1] > s for s in earlier))
    intervals = []
    start = 0            # the POV's own ring is visible
    is_open = True
    for d in range(1, L + 1):
        v = visible[d - 1]
        if is_open and not v:
            intervals.append((start, d))
            is_open = False
        elif not is_open and v:
            start = d
            is_open = True
    if is_open:
        intervals.append((start, L))
    return intervals


def measure(intervals: list[tuple[int, int]]) -> int:
    return sum(e * e - s * s for s, e in intervals)


def walk_limit(step: float, max_range: float, t: float) -> int:
    if not (max_range > 0) or math.isinf(max_range):
        return 1 << 62
    return int(math.floor(max_range / (step * math.sqrt(1.0 + t * t))))


def virtual_povs(view: View, t: float, i: int, j0: int) -> list[tuple[int, float]]:
    """[(b, weight)] of the sampled lines that straddle view cell (i, j0): the
    line through i + r(j0) (weight 1 - r) and the one through i - 1 + r(j0)
    (weight r), as Kernel-3 (Alg. 9) blends them."""
    y = j0 * t
    dest = math.floor(y)
    r = y - dest
    if r == 0.0:
        return [(i - dest, 1.0)]
    if r < AMBIGUOUS or 1 - r < AMBIGUOUS:
        raise AssertionError("fraction too close to 0 or 1 for a float reference")
    hi_ok = i <= view.H - 2
    lo_ok = i >= 1
    if hi_ok and lo_ok:
        return [(i - dest, 1.0 - r), (i - dest - 1, r)]
    if hi_ok:
        return [(i - dest, 1.0)]
    return [(i - dest - 1, 1.0)]


def cell_direction_cv(dem: np.ndarray, step: float, h0: float, n: int, max_range: float,
                      iD: int, jD: int, k: int) -> list[dict]:
    frame, m = frame_of(n, k)
    t = tan_of(n, m)
    view = View(dem, frame)
    i, j0 = view.cell_to_view(iD, jD)
    K = walk_limit(step, max_range, t)
    res = []
    for b, w in virtual_povs(view, t, i, j0):
        h = _height(view.V, b + j0 * t, j0) + h0
        pf = line_profile(view, t, j0, b, +1, K)
        pb = line_profile(view, t, j0, b, -1, K)
        res.append(dict(w=w, cv_fwd=measure(visible_intervals(h, pf)),
                        cv_bwd=measure(visible_intervals(h, pb)), L_fwd=len(pf), L_bwd=len(pb)))
    return res


def brute_total_viewshed(dem: np.ndarray, step: float, h0: float, n: int, max_range: float = 0.0,
                         cells=None) -> np.ndarray:
    rows, cols = dem.shape
    if cells is None:
        cells = range(rows * cols)
    out = []
    for c in cells:
        iD, jD = divmod(int(c), cols)
        acc = 0.0
        for k in range(n):
            frame, m = frame_of(n, k)
            t = tan_of(n, m)
            g = 1.0 + t * t
            part = sum(v["w"] * (v["cv_fwd"] + v["cv_bwd"])
                       for v in cell_direction_cv(dem, step, h0, n, max_range, iD, jD, k))
            acc += g * part
        out.append(math.pi / (2 * n) * step * step * acc)
    return np.array(out)


def walk_lengths(rows: int, cols: int, n: int, step: float, max_range: float, iD: int, jD: int, k: int):
    """[(weight, L_fwd, L_bwd, g)] for cell (iD, jD) and direction k (flat terrain)."""
    dem = np.zeros((rows, cols), np.float32)
    frame, m = frame_of(n, k)
    t = tan_of(n, m)
    return [(v["w"], v["L_fwd"], v["L_bwd"], 1.0 + t * t)
            for v in cell_direction_cv(dem, step, 1.0, n, max_range, iD, jD, k)]


def direct_profile(view: View, t: float, i: int, j0: int, direction: int, K: int) -> list[float]:
    """Heights of the targets of the half-line through view cell (i, j0)
    itself (no virtual POVs): Y(j) = i + (j - j0) * t."""
    out = []
    d = 1
    while d <= K:
        j = j0 + direction * d
        if j < 0 or j >= view.W:
            break
        Y = i + (j - j0) * t
        if 0 < abs(Y - round(Y)) < AMBIGUOUS:
            raise AssertionError("sample too close to a grid line for a float reference")
        if not _usable(view.H, Y):
            break
        out.append(_height(view.V, Y, j))
        d += 1
    return out


def brute_direct_viewshed(dem: np.ndarray, step: float, h0: float, n: int, max_range: float = 0.0,
                          cells=None) -> np.ndarray:
    """Singular viewsheds by definition (Alg. 1-3): the POV is the cell itself
    and every line of sight passes through it."""
    rows, cols = dem.shape
    if cells is None:
        cells = range(rows * cols)
    out = []
    for c in cells:
        iD, jD = divmod(int(c), cols)
        acc = 0.0
        for k in range(n):
            frame, m = frame_of(n, k)
            t = tan_of(n, m)
            view = View(dem, frame)
            i, j0 = view.cell_to_view(iD, jD)
            K = walk_limit(step, max_range, t)
            h = float(view.V[i, j0]) + h0
            cv = sum(measure(visible_intervals(h, direct_profile(view, t, i, j0, s, K))) for s in (+1, -1))
            acc += (1.0 + t * t) * cv
        out.append(math.pi / (2 * n) * step * step * acc)
    return np.array(out)


def sector_of(n: int, di: int, dj: int) -> tuple[int, float]:
    """Half-line sector k' (0..2n-1) nearest to the direction (di south, dj
    east) and the fraction of q = atan2(di, dj) n / pi (ties at 0.5)."""
    q = math.atan2(di, dj) * n / math.pi
    kp = math.floor(q + 0.5) % (2 * n)
    return kp, q - math.floor(q)


def brute_visibility_map(dem: np.ndarray, step: float, h0: float, n: int, povs, max_range: float = 0.0):
    """Visibility counts by rescanning: a cell is seen from a POV when the
    target at its walk-axis column on its sector's half-line through the POV
    is strictly above every earlier target's slope."""
    rows, cols = dem.shape
    count = np.zeros((rows, cols), np.int32)
    for (i0, j0) in povs:
        for iD in range(rows):
            for jD in range(cols):
                if (iD, jD) == (i0, j0):
                    count[iD, jD] += 1
                    continue
                kp, _ = sector_of(n, iD - i0, jD - j0)
                k = kp % n
                frame, m = frame_of(n, k)
                t = tan_of(n, m)
                view = View(dem, frame)
                vi0, vj0 = view.cell_to_view(i0, j0)
                vi, vj = view.cell_to_view(iD, jD)
                plus = (frame <= 1) == (kp < n)
                d = (vj - vj0) if plus else (vj0 - vj)
                if d < 1:
                    continue
                prof = direct_profile(view, t, vi0, vj0, 1 if plus else -1, walk_limit(step, max_range, t))
                if d > len(prof):
                    continue
                h = float(view.V[vi0, vj0]) + h0
                slopes = [(prof[x] - h) / (x + 1) for x in range(d)]
                if all(slopes[d - 1] > s for s in slopes[: d - 1]):
                    count[iD, jD] += 1
    return count

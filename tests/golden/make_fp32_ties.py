"""Writes fp32_ties.txt: near-tie lines of sight whose measures depend on the
exact order of the single-precision operations of the FP32-decision reading.

That reading (the paper declares heights and slopes "float" in Alg. 6, 7 and
8) forms, for a sample of a line blending view rows a and a + 1 with the
fraction fr of Alg. 6,

    r  = float(fr) * 2^-32          (exact scaling of a rounded integer)
    wa = fl(1 - r)
    z  = fl(fl(wa * va) + fl(r * vb))        (z = va when fr = 0)
    h  = fl(z_pov + float(h0))
    th = fl(fl(z - h) * fl(1 / d))

and decides "visible" iff th is strictly above the running maximum (Alg. 8),
a segment closing with d^2 - open^2 (visible at the start, above
recomputed per target, the open segment closed at the last target).
The FP64 reading takes the same steps in double precision with a true
division, r = fr / 2^32 exactly and h0 unrounded.

Everything here is exact rational arithmetic (fractions.Fraction) with an
explicit round-to-nearest-even to 24 or 53 significand bits; it shares no code
with the oracle.  The lines are the direction k = 1 of n = 8 (22.5 degrees,
identity view), whose samples blend two DEM rows; the DEM values are chosen
so that the targets of a POV are nearly collinear, which makes almost every
decision a near-tie.  The script keeps cases until each of these plausible
mistakes in the FP32 reading changes at least one expected measure:

    div : th = fl(fl(z - h) / d)               (a division, not fl(1/d))
    fma : z = fl(wa * va + fl(r * vb))         (a fused multiply-add)
    h64 : h = fl(z_pov + h0)                   (h0 not rounded first)
    w64 : wa = fl(1 - fr / 2^32)               (the weight from the exact r)

Run it from the repository root: python tests/golden/make_fp32_ties.py
"""
from __future__ import annotations

import math
import os
import random
from fractions import Fraction as Q

HERE = os.path.dirname(os.path.abspath(__file__))
N, K = 8, 1                 # direction 1 of 8: alpha = pi / 8, identity view
ROWS, COLS = 4, 8           # line b = 0 stays inside the DEM at every column
TWO32 = 1 << 32


def rnd(x: Q, bits: int) -> Q:
    """x rounded to the nearest value with `bits` significand bits (ties to
    even); normal range only."""
    if x == 0:
        return Q(0)
    s = -1 if x < 0 else 1
    a = abs(x)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Q(2) ** e > a:
        e -= 1
    ulp = Q(2) ** (e - bits + 1)
    q, rem = divmod(a, ulp)
    if rem * 2 > ulp or (rem * 2 == ulp and q % 2 == 1):
        q += 1
    return s * q * ulp


def f32(x: Q) -> Q:
    return rnd(x, 24)


def f64(x: Q) -> Q:
    return rnd(x, 53)


def t_fx() -> int:
    # llround(tan(alpha) * 2^32), as the direction table rounds it
    return int(math.floor(math.tan(math.pi * (2 * K) / (2.0 * N)) * TWO32 + 0.5))


TFX = t_fx()


def sample(dem, j, prec, mut):
    """Height of the sample of line b = 0 at column j."""
    y = j * TFX
    a, fr = y >> 32, y & (TWO32 - 1)
    va, vb = dem[a][j], dem[a + 1][j] if fr else None
    if fr == 0:
        return va
    if prec == 64:
        r = Q(fr, TWO32)
        return f64(f64(f64(1 - r) * va) + f64(r * vb))
    r = f32(Q(fr)) / TWO32
    wa = f32(1 - Q(fr, TWO32)) if mut == "w64" else f32(1 - r)
    if mut == "fma":
        return f32(wa * va + f32(r * vb))
    return f32(f32(wa * va) + f32(r * vb))


def walk(dem, j0, step, prec, h0, mut):
    rd = f64 if prec == 64 else f32
    zp = sample(dem, j0, prec, mut)
    if prec == 64:
        h = f64(zp + h0)
    else:
        h = f32(zp + h0) if mut == "h64" else f32(zp + f32(h0))
    vis, opn, last, cv = True, 0, 0, 0
    mx = None
    dd = 1
    while 0 <= j0 + step * dd < COLS:
        z = sample(dem, j0 + step * dd, prec, mut)
        diff = rd(z - h)
        if prec == 64:
            th = f64(diff / dd)
        elif mut == "div":
            th = f32(diff / dd)
        else:
            th = f32(diff * f32(Q(1, dd)))
        above = mx is None or th > mx
        if above and not vis:
            opn = dd
        if not above and vis:
            cv += dd * dd - opn * opn
        vis = above
        if mx is None or th > mx:
            mx = th
        last = dd
        dd += 1
    if vis:
        cv += last * last - opn * opn
    return cv


def line_cv(dem, prec, h0, mut=None):
    return [walk(dem, j, +1, prec, h0, mut) + walk(dem, j, -1, prec, h0, mut) for j in range(COLS)]


def candidate(rng: random.Random):
    """Rows a and a + 1 of every column hold nearly the same value, so the
    blended heights lie close to a line of slope s above the POV at j = 0.
    Small ground heights make h = z + h0 round on a fine grid, where rounding
    h0 first can move it."""
    # the observer height as the double the oracle receives
    h0 = Q(rng.choice([0.1, 1.7, 2.3, 7.0 / 3.0]))
    base = f32(Q(rng.randint(1, 4000), 1 << rng.choice([3, 10, 14])))
    s = Q(rng.randint(-400, 400), 97 * rng.choice([1, 64]))
    dem = [[Q(0)] * COLS for _ in range(ROWS)]
    for j in range(COLS):
        a = (j * TFX) >> 32
        v = f32(base + h0 + s * j) if j else base
        for i in range(ROWS):
            dem[i][j] = f32(v + Q(rng.randint(-40, 40), 1 << 22) * (1 + abs(v)))
        dem[a][j] = v
        dem[a + 1][j] = f32(v + Q(rng.randint(-3, 3), 1 << 23) * (1 + abs(v)))
    return dem, h0


def screen(dem, h0):
    """A fast float32 / float64 pass (numpy) that picks candidates worth the
    exact derivation; it decides nothing that is stored."""
    import numpy as np
    f = np.float32
    d32 = [[f(float(v)) for v in row] for row in dem]
    h0f = float(h0)

    def samp(j, mode):
        y = j * TFX
        a, fr = y >> 32, y & (TWO32 - 1)
        if fr == 0:
            return float(d32[a][j]) if mode == 64 else d32[a][j]
        if mode == 64:
            r = fr / TWO32
            return (1.0 - r) * float(d32[a][j]) + r * float(d32[a + 1][j])
        r = f(fr) * f(2.0 ** -32)
        wa = f(1.0 - fr / TWO32) if mode == "w64" else f(1.0) - r
        if mode == "fma":
            return f(float(wa) * float(d32[a][j]) + float(r * d32[a + 1][j]))
        return wa * d32[a][j] + r * d32[a + 1][j]

    def cvs(mode):
        out = []
        for j0 in range(COLS):
            zp = samp(j0, mode)
            if mode == 64:
                h = zp + h0f
            elif mode == "h64":
                h = f(float(zp) + h0f)
            else:
                h = zp + f(h0f)
            tot = 0
            for st in (1, -1):
                vis, opn, last, cv, mx, dd = True, 0, 0, 0, None, 1
                while 0 <= j0 + st * dd < COLS:
                    z = samp(j0 + st * dd, mode)
                    if mode == 64:
                        th = (z - h) / dd
                    elif mode == "div":
                        th = (z - h) / f(dd)
                    else:
                        th = (z - h) * (f(1.0) / f(dd))
                    ab = mx is None or th > mx
                    if ab and not vis:
                        opn = dd
                    if not ab and vis:
                        cv += dd * dd - opn * opn
                    vis = ab
                    mx = th if mx is None or th > mx else mx
                    last = dd
                    dd += 1
                if vis:
                    cv += last * last - opn * opn
                tot += cv
            out.append(tot)
        return out

    base = cvs(32)
    return base != cvs(64), {m: cvs(m) != base for m in ("div", "fma", "h64", "w64")}


def main():
    rng = random.Random(2003022000)
    muts = ["div", "fma", "h64", "w64"]
    caught = {m: 0 for m in muts}
    kept = []
    tries = 0
    while (len(kept) < 4 or min(caught.values()) == 0) and tries < 200000:
        tries += 1
        dem, h0 = candidate(rng)
        d64, dm = screen(dem, h0)
        if not d64 or not any(d and caught[m] < 2 for m, d in dm.items()):
            continue
        c32 = line_cv(dem, 32, h0)
        c64 = line_cv(dem, 64, h0)
        diffs = {m: line_cv(dem, 32, h0, m) != c32 for m in muts}
        if c32 == c64 or not any(d and caught[m] < 2 for m, d in diffs.items()):
            continue
        for m, d in diffs.items():
            caught[m] += int(d)
        kept.append((dem, h0, c32, c64, [m for m, d in diffs.items() if d]))
    assert min(caught.values()) > 0, f"no case catches every mistake: {caught}"
    lines = [
        "# Near-tie lines of sight pinning the oracle's FP32-decision mode (prec=32)",
        "# against exact rational arithmetic; written by make_fp32_ties.py (see its",
        "# docstring for the operation order).",
        f"# Every case: direction k = {K} of n = {N}, DEM {ROWS} x {COLS}, step 1, no range,",
        "# line b = 0; h0 (a double) and the dem rows (float32 values) are in hex;",
        "# cv32 / cv64 are the forward + backward measures of the POVs j = 0 .. 7",
        "# in the FP32 and FP64",
        "# readings; 'catches' lists the planted mistakes that change cv32.",
        f"t_fx {TFX}",
    ]
    for dem, h0, c32, c64, cat in kept:
        lines.append(f"case h0 {float(h0).hex()}")
        for row in dem:
            lines.append("row " + " ".join(float(v).hex() for v in row))
        lines.append("cv32 " + " ".join(map(str, c32)))
        lines.append("cv64 " + " ".join(map(str, c64)))
        lines.append("catches " + (" ".join(cat) if cat else "-"))
    with open(os.path.join(HERE, "fp32_ties.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")
    print(f"{len(kept)} cases after {tries} candidates; mistakes caught: {caught}")


if __name__ == "__main__":
    main()

"""The tile binning's FP32 row rule, restated in numpy for the checks of the
tile lists.

A surfel is listed in tile (tx, ty) when, in the band of pixel rows of tile
row ty, the pixel columns its footprint may reach (the ellipse
{rho_obj <= rho_max} united with the screen-filter disk, each side widened by
a rounding margin) fall in tile column tx.  The CUDA path evaluates this rule
in FP32 with explicit round-to-nearest operations on the stored footprint
shape (gs_frame_copy_cover); here every operation is the same IEEE binary32
operation: numpy's float32 add, subtract, multiply and square root are
correctly rounded, and a fused multiply-add (one rounding of a b + c) is
reconstructed exactly from float64 (fma32).  So the instances this module
lists must equal the GPU's bit for bit, and the checks can then rebuild the
sorted lists and ranges independently of the CUDA sort.
"""
import numpy as np

F = np.float32
TILE = 16


def fma32(a, b, c):
    """round_binary32(a * b + c) with one rounding, for float32 arrays.  The
    product of two float32 values is exact in float64; s + e = a b + c
    exactly by Knuth's TwoSum; rounding s to binary32 is then correct unless
    s lies exactly on a midpoint between two binary32 values, where the sign
    of e decides."""
    a = np.asarray(a, np.float32).astype(np.float64)
    b = np.asarray(b, np.float32).astype(np.float64)
    c = np.asarray(c, np.float32).astype(np.float64)
    p = a * b
    s = p + c
    bb = s - p
    e = (p - (s - bb)) + (c - bb)
    r = s.astype(np.float32)
    up = np.nextafter(s, np.inf).astype(np.float32)
    dn = np.nextafter(s, -np.inf).astype(np.float32)
    mid = up != dn
    return np.where(mid & (e > 0), up, np.where(mid & (e < 0), dn, r)).astype(np.float32)


def unpack(geom_words):
    """[n][14] int32 words -> dict of float32 fields and int32 boxes."""
    w = np.ascontiguousarray(np.asarray(geom_words, np.int32))
    f = w[:, :10].view(np.float32)
    names = ["cx_hi", "cx_lo", "cy_hi", "cy_lo", "e0x", "e0y", "hy", "t", "slope", "wsc"]
    g = {k: f[:, i].copy() for i, k in enumerate(names)}
    for i, k in enumerate(["ilo", "ihi", "jlo", "jhi"]):
        g[k] = w[:, 10 + i].astype(np.int64)
    return g


def band_pixels(g, ja, jb, rf):
    """Pixel columns [ilo, ihi] reached in pixel rows ja..jb (arrays), and
    whether there are any."""
    rf = F(rf)
    ja = np.maximum(ja, g["jlo"])
    jb = np.minimum(jb, g["jhi"])
    ok = ja <= jb
    one_em5, one_em3 = F(1e-5), F(1e-3)
    ya = (((ja.astype(F) + F(0.5)) - g["cy_hi"]) - g["cy_lo"]).astype(F)
    yb = (((jb.astype(F) + F(0.5)) - g["cy_hi"]) - g["cy_lo"]).astype(F)
    my = fma32(one_em5, np.abs(ya) + np.abs(yb), one_em3)
    n = ya.shape[0]
    lo = np.full(n, np.inf, F)
    hi = np.full(n, -np.inf, F)
    hy, e0x, e0y, t, slope, wsc = g["hy"], g["e0x"], g["e0y"], g["t"], g["slope"], g["wsc"]
    with np.errstate(invalid="ignore", over="ignore"):
        dya = ya - e0y
        dyb = yb - e0y
        ell = (hy > 0) & (dyb >= -(hy + my)) & (dya <= hy + my)
        yr = np.fmin(np.fmax(t, dya), dyb)
        yl = np.fmin(np.fmax(-t, dya), dyb)
        qr = np.fmax((hy - yr) * (hy + yr), F(0))
        ql = np.fmax((hy - yl) * (hy + yl), F(0))
        ehi = fma32(wsc, np.sqrt(qr), fma32(slope, yr, e0x))
        elo = fma32(-wsc, np.sqrt(ql), fma32(slope, yl, e0x))
        ms = np.abs(slope) * my
        hi = np.where(ell, ehi + ms, hi).astype(F)
        lo = np.where(ell, elo - ms, lo).astype(F)
        yn = np.fmin(np.fmax(F(0), ya), yb)
        r2 = rf * rf - yn * yn
        disk = r2 >= -((F(2) * rf) * my)
        h = np.sqrt(np.fmax(r2, F(0))) + my
        lo = np.where(disk, np.fmin(lo, -h), lo).astype(F)
        hi = np.where(disk, np.fmax(hi, h), hi).astype(F)
        ok &= lo <= hi
        m = fma32(one_em5, np.abs(lo) + np.abs(hi), one_em3)
        xlo = (g["cx_hi"] + (lo - m)) + g["cx_lo"]
        xhi = (g["cx_hi"] + (hi + m)) + g["cx_lo"]
        ilo = np.ceil(np.fmax(xlo, F(-1)) - F(0.5))
        ihi = np.floor(np.fmin(xhi, F(1e9)) - F(0.5))
    ilo = np.where(ok, ilo, 0).astype(np.int64)
    ihi = np.where(ok, ihi, -1).astype(np.int64)
    ilo = np.maximum(ilo, g["ilo"])
    ihi = np.minimum(ihi, g["ihi"])
    return ilo, ihi, ok & (ilo <= ihi)


def instances(geom_words, surfels, tiles_x, rf):
    """(surfel, tile) instances of the given surfels by the row rule, as two
    int64 arrays, in no particular order."""
    g_all = unpack(geom_words)
    surfels = np.asarray(surfels, np.int64)
    g = {k: v[surfels] for k, v in g_all.items()}
    ty0 = g["jlo"] // TILE
    ty1 = g["jhi"] // TILE + 1
    nrows = np.maximum(ty1 - ty0, 0)
    rep = np.repeat(np.arange(surfels.size), nrows)
    off = np.arange(rep.size) - np.repeat(np.cumsum(nrows) - nrows, nrows)
    ty = ty0[rep] + off
    gr = {k: v[rep] for k, v in g.items()}
    ilo, ihi, ok = band_pixels(gr, ty * TILE, ty * TILE + TILE - 1, rf)
    tx0 = np.where(ok, ilo // TILE, 0)
    tx1 = np.where(ok, ihi // TILE + 1, 0)
    ncol = tx1 - tx0
    rep2 = np.repeat(np.arange(rep.size), ncol)
    off2 = np.arange(rep2.size) - np.repeat(np.cumsum(ncol) - ncol, ncol)
    tile = ty[rep2] * tiles_x + tx0[rep2] + off2
    return surfels[rep[rep2]], tile


def sorted_lists(surf, tile, depth_bits, ntiles):
    """Stable order by (tile, FP32 depth bits, surfel index) and the per-tile
    ranges [start, end) (0, 0 for empty tiles), as the CUDA path's lists."""
    order = np.lexsort((surf, depth_bits[surf], tile))
    vals = surf[order]
    t = tile[order]
    ranges = np.zeros((ntiles, 2), np.int64)
    if t.size:
        present = np.unique(t)
        ranges[present, 0] = np.searchsorted(t, present, side="left")
        ranges[present, 1] = np.searchsorted(t, present, side="right")
    return vals, ranges

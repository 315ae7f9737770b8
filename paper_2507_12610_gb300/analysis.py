"""Statistics of particle states for the long-run checks (host side, numpy).

Angle of repose of a quasi-2D heap (Sec. 5, the piling example: mu_eff =
tan theta), packing fraction in a region, and kinetic energy.  Nothing here
is on the time-step path.
"""
from __future__ import annotations

import math

import numpy as np


def kinetic_energy(R, v, w, rho):
    """Translational and rotational kinetic energy of solid spheres (J)."""
    R = np.asarray(R, dtype=np.float64)
    m = 4.0 / 3.0 * math.pi * rho * R ** 3
    inertia = 0.4 * m * R ** 2
    et = 0.5 * float(np.sum(m * np.einsum("ij,ij->i", v, v)))
    er = 0.5 * float(np.sum(inertia * np.einsum("ij,ij->i", w, w)))
    return et, er


def surface_profile(x, z, R, lo, hi, width):
    """Free-surface height per bin along x: the highest sphere top (z + R) of
    the spheres whose centres fall in each bin of the given width; NaN where
    a bin is empty.  Returns (bin centres, heights)."""
    nb = int(math.ceil((hi - lo) / width))
    idx = np.floor((np.asarray(x) - lo) / width).astype(np.int64)
    ok = (idx >= 0) & (idx < nb)
    top = np.full(nb, -np.inf)
    np.maximum.at(top, idx[ok], (np.asarray(z) + np.asarray(R))[ok])
    top[~np.isfinite(top)] = np.nan
    return lo + (np.arange(nb) + 0.5) * width, top


def repose_angle(x, z, R, lo, hi, width, lo_frac=0.2, hi_frac=0.8):
    """Angle of repose of a heap from its surface profile.

    The two flanks are the profile bins left and right of the apex whose
    heights lie between lo_frac and hi_frac of the apex height (so the
    rounded apex and the curved bottom ends are left out); a least-squares
    line through each gives its slope.  Returns dict with the angles of the
    left and right flanks and their mean, in degrees, and the apex height.
    """
    xc, h = surface_profile(x, z, R, lo, hi, width)
    good = np.isfinite(h)
    if good.sum() < 5:
        raise ValueError("no heap")
    xc, h = xc[good], h[good]
    k = int(np.argmax(h))
    H = float(h[k])
    out = {"apex_height": H, "apex_x": float(xc[k])}
    for side, sel in (("left", np.arange(k + 1)), ("right", np.arange(k, len(h)))):
        xs, hs = xc[sel], h[sel]
        band = (hs >= lo_frac * H) & (hs <= hi_frac * H)
        if band.sum() < 3:
            out[side] = float("nan")
            continue
        slope = np.polyfit(xs[band], hs[band], 1)[0]
        out[side] = math.degrees(math.atan(abs(slope)))
    out["mean"] = 0.5 * (out["left"] + out["right"])
    return out


def drum_surface_angle(x, R, drum_radius, drum_length, width, band=0.5, section=0.5):
    """Free-surface angle of the bed in a drum turning about the x axis.

    The spheres of the middle `section` of the drum's length (away from the
    end caps) are projected onto the y-z cross-section; the surface profile
    is the highest sphere top (z + R) per bin of the given width along y, and
    a least-squares line through the bins with |y| < band * drum_radius
    (away from the shell) gives its slope.  Returns the angle to the
    horizontal in degrees (positive: the surface rises towards +y).
    """
    x = np.asarray(x)
    sel = np.abs(x[:, 0]) < 0.5 * section * drum_length
    half = band * drum_radius
    yc, h = surface_profile(x[sel, 1], x[sel, 2], np.asarray(R)[sel], -half, half, width)
    good = np.isfinite(h)
    if good.sum() < 4:
        raise ValueError("no free surface")
    slope = np.polyfit(yc[good], h[good], 1)[0]
    return math.degrees(math.atan(slope))


def packing_fraction(x, R, box_lo, box_hi):
    """Solid fraction of an axis-aligned box: volume of the spheres whose
    centres lie inside it over its volume (spheres cut by the box faces are
    counted whole or not at all, which averages out for boxes much larger
    than a sphere)."""
    x = np.asarray(x)
    lo, hi = np.asarray(box_lo, dtype=np.float64), np.asarray(box_hi, dtype=np.float64)
    inside = np.all((x >= lo) & (x < hi), axis=1)
    vol = float(np.prod(hi - lo))
    return float(np.sum(4.0 / 3.0 * math.pi * np.asarray(R)[inside] ** 3)) / vol


def heap_core_fraction(x, R, gap, apex_height, apex_x, theta_deg, margin):
    """Packing fraction in the core of a quasi-2D heap: the full gap across,
    a box centred under the apex from `margin` above the floor to 40 % of the
    apex height, as wide as the heap at that height minus `margin` each side."""
    z1 = 0.4 * apex_height
    half = (apex_height - z1) / math.tan(math.radians(theta_deg)) - margin
    if half <= 0:
        raise ValueError("heap too small for a core region")
    lo = (apex_x - half, -0.5 * gap, margin)
    hi = (apex_x + half, 0.5 * gap, z1)
    return packing_fraction(x, R, lo, hi)

"""Closed forms that the tests compare the oracle and the CUDA path against.

Written from the paper's formulas and from the mathematics; nothing here calls the
oracle or the CUDA library.
"""
import math

from scipy.integrate import quad


def inclined_disk_p(incl, kz2=0.0):
    """Degree of linear polarization Q/I of the inclined-disk test (Sec. 3.1).

    Light travelling in the disk plane, isotropic in azimuth, scattered once by
    dipole (Rayleigh) grains and seen at inclination i has p = sin^2 i / (2 + sin^2 i),
    polarized along the projected disk axis (Q > 0 in the camera basis e_y = -theta-hat).

    Derivation (used here with a small out-of-plane part): the scattered field is the
    incident field projected on the plane normal to the line of sight o, so an
    unpolarized beam along k adds (1 - k k^T)/2, projected, to the coherency matrix.
    Summed over the beams with their weights, only M = <k k^T> enters; by the disk's
    symmetry M = diag(a, a, c) with c = ``kz2`` = <k_z^2> and a = (1 - c)/2.  In the
    image basis e_x = y-hat, e_y = (-cos i, 0, sin i) of o = (sin i, 0, cos i):
    C_xx = (1 - a)/2, C_yy = ((1 - a) cos^2 i + (1 - c) sin^2 i)/2, I = C_xx + C_yy,
    Q = C_yy - C_xx.  With c = 0 this is the paper's formula.
    """
    c = float(kz2)
    a = 0.5 * (1.0 - c)
    s2, c2 = math.sin(incl) ** 2, math.cos(incl) ** 2
    return (a - c) * s2 / ((1.0 - a) * (1.0 + c2) + (1.0 - c) * s2)


def thin_annulus_kz2(h, r_in, r_out):
    """<k_z^2> of the light a central isotropic point source sends through a uniform
    annulus r_in <= R <= r_out, |z| <= h, weighted by the path length inside it (the
    weight every segment carries in the step-1 tally of an optically thin medium).
    A ray of direction cosine s = |n_z| runs inside from t = r_in / sqrt(1 - s^2) to
    min(r_out / sqrt(1 - s^2), h / s)."""

    def length(s):
        cb = math.sqrt(1.0 - s * s)
        t1 = r_out / cb if s == 0.0 else min(r_out / cb, h / s)
        return max(0.0, t1 - r_in / cb)

    s_out = h / math.hypot(h, r_out)
    s_in = h / math.hypot(h, r_in)
    num = quad(lambda s: s * s * length(s), 0.0, s_out)[0] + quad(lambda s: s * s * length(s), s_out, s_in)[0]
    den = quad(length, 0.0, s_out)[0] + quad(length, s_out, s_in)[0]
    return num / den

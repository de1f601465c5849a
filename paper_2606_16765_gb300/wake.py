"""Wake diagnostics from the obstacle force record (host post-processing of
what the solver's force epilogue writes; no lattice arithmetic).

  Strouhal number  St = f D / U, f the dominant frequency of the lift F_y(t)
                   (periodogram of the mean-removed, Hann-windowed signal,
                   peak refined by a parabola through the log-power of the
                   three bins around it).
  Drag coefficient C_d = 2 <F_x> / (rho U^2 A), A the projected area (D times
                   the span for a spanwise cylinder).
  Recirculation    l_r: distance from the rear of the body to the end of the
  length           backflow region of the mean streamwise velocity on the
                   wake centreline (first zero up-crossing, linear
                   interpolation between cells).

The paper reports the Strouhal number of the wake (Sec. 3.3, vertical
velocity spectrum) and drag coefficients (Sec. 3.3, Table 1) as its validation
measures; these helpers compute them from the momentum-exchange force.
"""
from __future__ import annotations

import numpy as np


def dominant_frequency(signal, dt=1.0, band=None):
    """Frequency (cycles per unit of dt) of the largest non-zero periodogram
    peak of a real signal, optionally searched only inside band = (lo, hi)."""
    x = np.asarray(signal, dtype=np.float64)
    n = len(x)
    if n < 8:
        raise ValueError("signal too short")
    w = np.hanning(n)
    p = np.abs(np.fft.rfft((x - x.mean()) * w)) ** 2
    freq = np.arange(len(p)) / (n * dt)
    sel = np.ones(len(p), bool)
    sel[0] = False
    if band is not None:
        sel &= (freq >= band[0]) & (freq <= band[1])
    if not sel.any():
        raise ValueError("no frequency bin inside the band")
    k = int(np.argmax(np.where(sel, p, -1.0)))
    shift = 0.0
    if 1 <= k < len(p) - 1 and p[k - 1] > 0 and p[k + 1] > 0:
        a, b, c = np.log(p[k - 1]), np.log(p[k]), np.log(p[k + 1])
        den = a - 2 * b + c
        if den != 0:
            shift = 0.5 * (a - c) / den
    return (k + shift) / (n * dt)


def strouhal(lift, d, u, every=1, st_band=None):
    """St of a lift record sampled every `every` steps, diameter d and inlet
    speed u in lattice units; st_band = (lo, hi) limits the search to a range
    of St (e.g. to keep a channel's acoustic modes, St = d c_s / (2 H u) and
    above, out of a shedding measurement)."""
    band = None if st_band is None else (st_band[0] * u / d, st_band[1] * u / d)
    return dominant_frequency(lift, dt=float(every), band=band) * d / u


def drag_coefficient(fx, d, span, u, rho=1.0):
    """C_d from the mean streamwise force over a record."""
    return 2.0 * float(np.mean(fx)) / (rho * u * u * d * span)


def recirculation_length(u_line, x_rear):
    """l_r in cells from the mean streamwise velocity u_line[x] along the wake
    centreline: the first x > x_rear where u crosses zero upwards after a
    backflow (u < 0) region that starts behind x_rear, minus x_rear (the x of
    the body's rear surface).  0 when there is no backflow."""
    u = np.asarray(u_line, dtype=np.float64)
    start = int(np.floor(x_rear)) + 1
    neg = np.nonzero(u[start:] < 0)[0]
    if len(neg) == 0:
        return 0.0
    k = start + int(neg[0])
    while k + 1 < len(u) and u[k + 1] < 0:
        k += 1
    if k + 1 >= len(u):
        return float(len(u) - 1 - x_rear)
    x0 = k + u[k] / (u[k] - u[k + 1])            # u[k] < 0 <= u[k+1]
    return float(x0 - x_rear)

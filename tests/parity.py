"""Shared parity rules for the GPU tests (no library code here).

Tolerances (the FFT rounding is relative to the largest value of the
convolved window, O(K) near the divider, hence the absolute floor in K):
  FP64 methods (FFT_FP64, STENCIL_FP64) and the doubled-FP32 ones (FFT_DF32,
  STENCIL_DF32):
      |gpu - oracle| <= 1e-10 |oracle| + 1e-12 K
  FP32-split FFT:
      |gpu - oracle| <= FP32_REL |oracle| + FP32_ABS K
Boundary rows may differ from the oracle only where the oracle's margin
|continuation - exercise| at the divider is within the tie band of the method.
FP64 methods may then move the divider by one cell.  The FP32-split method may
move it further: continuation and exercise value meet tangentially at the
exercise boundary (smooth pasting), so a value error of FP32 size shifts the
crossing by about sqrt(error / curvature) cells, which at small margins spans
several cells; each such row must still lie inside the FP32 tie band.  The
doubled-FP32 stencil carries the rounding of every row (at most ~2^-47 of the
value per row, the weights summing to at most 1: below 6e-11 of the value at
T <= 8192), so its tie band is 100 times the FP64 one, still one cell of reach.
"""
import numpy as np

import oracle

FP64_REL = 1e-10
FP64_ABS = 1e-12
FP32_REL = 2e-6
FP32_ABS = 2e-6


def price_tol(method, price_ref, K):
    if method == 1:
        return FP32_REL * abs(price_ref) + FP32_ABS * K
    return FP64_REL * abs(price_ref) + FP64_ABS * K


def tie_band(method, req):
    base = oracle.tie_band(req)
    if method == 1:
        return base * 1e6
    if method == 4:
        return base * 100
    return base


def check_boundary(method, req, got, want, margin):
    """Return the rows that differ outside the tie band."""
    got = np.asarray(got)
    want = np.asarray(want)
    diff = np.nonzero(got != want)[0]
    band = tie_band(method, req)
    reach = 1 if method != 1 else None
    bad = [int(i) for i in diff
           if not (margin[i] <= band and (reach is None or abs(int(got[i]) - int(want[i])) <= reach))]
    return bad, len(diff)

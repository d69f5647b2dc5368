"""Floating-point bars of the GPU parity tests (single precision vs the FP64 oracle).

FORWARD = 1e-4 (the transform bar, 0-255 scale): applied to each level's
coefficients divided by that level's DC gain (2^(j-1) for level j, 2^L for
the lowpass), the scale on which that level's numbers are pixels.

INVERSE = 1e-4: the inverse transform and the decoder's reconstructed planes
against the oracle's inverse of the same coefficients, max abs on the 0-255
scale.  The LP synthesis of levels 2..L computes in float-float, with the
CDF 9/7 taps held as float-float and the lowpass images between levels
stored as (hi, lo) pairs; level 1 runs in single precision centred on a
per-tile constant, which keeps its rounding at the scale of a tile's
deviation from its mean.  Measured 4.9e-5 (uniform noise), 5.9e-5 (integer
noise) and 2.1e-5 (smooth planes) at 1080p, 5 levels.

ROUND_TRIP = FORWARD + INVERSE: the GPU's inverse of its own forward
coefficients against the input carries both errors.
"""
FORWARD = 1e-4
INVERSE = 1e-4
ROUND_TRIP = FORWARD + INVERSE

# Gradients of the threshold-tuning loss mean((S soft_T(A x) - x)^2).  The
# residual r = S y - x carries the forward and inverse errors (at most
# ROUND_TRIP = 2e-4 absolute on the 0-255 scale), and every gradient entry is
# a sum of the adjoint image of 2r/N weighted by +-1 masks, so its relative
# error is about that absolute error over the typical residual size (a few
# units at thresholds of a few units): 2e-4 / 3 < 1e-4.  Coefficients within
# the forward error of their threshold may flip their mask; each flip moves
# one term of a sum over a whole subband.  The bar leaves a factor ten:
GRAD_REL = 1e-3

# Fixed-order single-precision sums of n terms (block partials of up to 4096
# terms, then a double-precision sum of the partials): error below
# (log2(4096) + 2) * 2^-24 * sum |terms| = 8.3e-7 * sum |terms|.
SUM_REL = 1e-5

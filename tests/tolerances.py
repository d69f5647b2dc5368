"""Floating-point bars of the GPU parity tests (single precision vs the FP64 oracle).

FORWARD = 1e-4 (the transform bar, 0-255 scale): applied to each level's
coefficients divided by that level's DC gain (2^(j-1) for level j, 2^L for
the lowpass), the scale on which that level's numbers are pixels.

inverse_bound(L, k) = L * FORWARD: the synthesis path (inverse transform,
decoder) computes with compensated (float-float) arithmetic inside every
kernel, so its error is the single-precision rounding of the values it
stores between launches, level by level.  Each level's reconstruction gets
the same per-level budget as the forward transform, and the output is the
sum of the L levels' reconstructions, so the budgets add.  Measured: 4e-5
(2 levels) to 1.2e-4 (5 levels, 1080p uniform-noise planes).
"""
FORWARD = 1e-4


def inverse_bound(levels, dirs_log2=None):
    return levels * FORWARD

# Gradients of the threshold-tuning loss mean((S soft_T(A x) - x)^2).  The
# residual r = S y - x carries the forward and inverse errors (at most
# FORWARD + inverse_bound(L) = (L + 1) * 1e-4 absolute on the 0-255 scale),
# and every gradient entry is a sum of the adjoint image of 2r/N weighted by
# +-1 masks, so its relative error is about that absolute error over the
# typical residual size (a few units at thresholds of a few units):
# (L + 1) * 1e-4 / 3 = 2e-4 at L = 5.  Coefficients within the forward error
# of their threshold may flip their mask; each flip moves one term of a sum
# over a whole subband.  The bar leaves a factor five:
GRAD_REL = 1e-3

# Fixed-order single-precision sums of n terms (block partials of up to 4096
# terms, then a double-precision sum of the partials): error below
# (log2(4096) + 2) * 2^-24 * sum |terms| = 8.3e-7 * sum |terms|.
SUM_REL = 1e-5

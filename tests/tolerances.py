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

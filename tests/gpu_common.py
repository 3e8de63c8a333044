"""Helpers for the GPU parity tests (inputs from synth, expected values from the oracle)."""
import numpy as np

import synth


def to_dev(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    return t.to("cuda", dtype=dtype) if dtype is not None else t.to("cuda")


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def rel_max(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


# (name, dims X Y Z T, bc, link roughness, coefficient record): sizes span several 32-site blocks
# and 128-site tiles with ragged tails, aliased offsets and antiperiodic boundaries.
SMALL_CASES = [
    ("4^3x8", (4, 4, 4, 8), (1, 1, 1, 1), 0.3, synth.placeholder_coeffs(1.0)),
    ("5^3x4-random-coeffs", (5, 5, 5, 4), (1, 1, 1, 1), 0.5, synth.random_coeffs(11)),
    ("3x5x4x3-antiperiodic-u0", (3, 5, 4, 3), (1, -1, 1, -1), 0.4, synth.random_coeffs(12, u0=0.87)),
    ("2x3x2x5-aliased", (2, 3, 2, 5), (-1, 1, 1, -1), 0.5, synth.random_coeffs(13)),
    ("7x6x5x9-ragged", (7, 6, 5, 9), (1, 1, 1, -1), 0.4, synth.random_coeffs(14)),
    ("4x4x5x4-kappa", (4, 4, 5, 4), (1, 1, 1, 1), 0.4, synth.random_coeffs(15).replace(kappa=0.11)),
    ("1x4x4x3-degenerate", (1, 4, 4, 3), (1, 1, 1, -1), 0.4, synth.random_coeffs(16)),
]
CASE_IDS = [c[0] for c in SMALL_CASES]

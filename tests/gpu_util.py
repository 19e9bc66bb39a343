"""Helpers for the GPU parity tests (no method arithmetic)."""
import numpy as np
import torch

import skygen


def rel_rms(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.sqrt(np.mean((a - b) ** 2) / np.mean(b ** 2)))


def max_rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b)) / np.sqrt(np.mean(b ** 2)))


def to_dev(sky, dev="cuda:0"):
    return {k: torch.from_numpy(np.ascontiguousarray(v)).to(dev) for k, v in sky.items()}


def sky(nside, lmax, pol=True, seeds=(0, 3, 1), b_scale=0.3, damp_t=100.0, damp_e=800.0):
    return skygen.make_sky(nside, lmax, pol, seeds[0], seeds[1], seeds[2], damp_t, damp_e,
                           b_scale=b_scale if pol else 0.0)

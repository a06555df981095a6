"""Helpers shared by the GPU parity tests (no method arithmetic here)."""
import json
import os

import numpy as np
import torch

# Acceptance bars for the fp32 CWT against the fp64 oracle (normwise).
CWT_REL_L2 = 1e-5
CWT_MAX_REL = 1e-4


def dev(x):
    return torch.as_tensor(x).to("cuda")


def cwt_errors(gpu, ref):
    g = gpu.astype(np.float64)
    rel_l2 = np.linalg.norm(g - ref) / np.linalg.norm(ref)
    max_rel = np.max(np.abs(g - ref)) / np.max(np.abs(ref))
    return rel_l2, max_rel


def random_box(n, L, seed, frac_out=0.02):
    """Uniform positions plus a few outside [0, L) and a few exactly on nodes."""
    rng = np.random.default_rng(seed)
    pos = rng.random((n, 3)) * L
    k = max(1, int(frac_out * n))
    pos[:k] += rng.choice([-L, L], size=(k, 3))
    pos[k:2 * k] = np.floor(pos[k:2 * k] / L * 8) * (L / 8)
    return pos.astype(np.float32)


def record(entry: dict):
    """Appends one JSON line of measured parity figures to the file named by
    the CWTHF_PRECISION_LOG environment variable (nothing when it is unset)."""
    path = os.environ.get("CWTHF_PRECISION_LOG")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps(entry, default=float) + "\n")

"""Helpers shared by the GPU parity tests (no K-Means arithmetic of the CUDA path here)."""
import numpy as np
import pytest
import torch

import oracle

# Assignment parity bar: identical wherever the oracle's top-2 gap exceeds
# 1e-6 * max(||x||^2, ||c_(1)||^2, ||c_(2)||^2).
GAP_REL = 1e-6


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")


def top2_index(X, C, chunk=1 << 16):
    """Index of the second-nearest centroid (numpy, chunked); used only to build the mask."""
    X = np.asarray(X, np.float64)
    C = np.asarray(C, np.float64)
    out = np.empty(X.shape[0], np.int64)
    for s in range(0, X.shape[0], chunk):
        x = X[s:s + chunk]
        dist = ((x[:, None, :] - C[None, :, :]) ** 2).sum(-1) if C.shape[0] * x.shape[0] < 3e7 else None
        if dist is None:
            dist = (x * x).sum(1)[:, None] - 2 * x @ C.T + (C * C).sum(1)[None, :]
        if C.shape[0] == 1:
            out[s:s + chunk] = 0
        else:
            out[s:s + chunk] = np.argpartition(dist, 1, axis=1)[:, 1]
    return out


def assignment_mask(X, C, rho_o, gap_o):
    """Rows where the assignment is unique enough to be compared exactly."""
    X = np.asarray(X, np.float64)
    C = np.asarray(C, np.float64)
    xn = (X * X).sum(1)
    cn = (C * C).sum(1)
    j2 = top2_index(X, C)
    scale = np.maximum(xn, np.maximum(cn[rho_o], cn[j2]))
    return gap_o > GAP_REL * scale, scale


def check_assignment(X, C, rho_gpu, name=""):
    """Compare a GPU assignment with the oracle's: exact on unmasked rows, near-optimal elsewhere."""
    rho_o, dmin_o, gap_o = oracle.assign(X, C)
    mask, scale = assignment_mask(X, C, rho_o, gap_o)
    rho_gpu = np.asarray(rho_gpu)
    bad = np.nonzero(mask & (rho_gpu != rho_o))[0]
    assert bad.size == 0, f"{name}: {bad.size} unmasked rows differ, e.g. {bad[:5]}"
    # masked rows: the chosen centroid is within the tolerance of the best one
    X64 = np.asarray(X, np.float64)
    C64 = np.asarray(C, np.float64)
    d_gpu = ((X64 - C64[rho_gpu]) ** 2).sum(1)
    assert np.all(d_gpu <= dmin_o + GAP_REL * scale + 1e-300), name
    return int((~mask).sum())


def rel_err(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))

"""Helpers shared by the GPU parity tests (test side only)."""
import math

import numpy as np

PHD, MUSIC, EV, MN = 0, 1, 2, 3
DB_TOL = 0.01          # pseudospectrum tolerance of the FP32 path, dB, over every grid point


def require_gpu():
    import pytest
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2007_14135_gb300 import build
    build.build()
    from paper_2007_14135_gb300 import doa
    return torch, doa


def factor_from_decomposition(evals, V, d, alg):
    """Factor B with B B^H = C of Table 3, formed from an eigendecomposition (test side).
    The tests check B B^H against the oracle's explicit C before they use B."""
    M = len(evals)
    En = V[:, d:]
    if alg == PHD:
        return V[:, -1:].copy()
    if alg == MUSIC:
        return En.copy()
    if alg == EV:
        return En / np.sqrt(evals[d:])[None, :]
    Pn = En @ En.conj().T
    return (Pn[:, 0] / Pn[0, 0].real)[:, None]


def db_error(P_gpu, P_ref):
    """max over k of |10 log10(P_gpu / P_ref)|."""
    P_gpu = np.asarray(P_gpu, np.float64)
    P_ref = np.asarray(P_ref, np.float64)
    return float(np.max(np.abs(10.0 * np.log10(P_gpu / P_ref))))


def percent_error(P_gpu, P_ref):
    """Eq. 4: 100/N sum |y_meas - y_gt| / |y_gt|."""
    P_gpu = np.asarray(P_gpu, np.float64)
    P_ref = np.asarray(P_ref, np.float64)
    return float(100.0 * np.mean(np.abs(P_gpu - P_ref) / np.abs(P_ref)))


def peak_margin(P, k):
    """Relative margin of a peak over its two grid neighbours: (P[k] - max(P[k-1], P[k+1])) / P[k]."""
    return float((P[k] - max(P[k - 1], P[k + 1])) / P[k])


def compare_peaks(idx_gpu, idx_ref, P_ref, bound):
    """True when the index sets agree, or every disagreement is a tie within `bound` (relative
    margin of the oracle's peak over its neighbours below the GPU's error bound)."""
    a, b = list(idx_gpu), list(idx_ref)
    if a == b:
        return True, []
    diff = sorted(set(a) ^ set(b))
    ties = [(k, peak_margin(P_ref, k)) for k in diff if 1 <= k < len(P_ref) - 1]
    return all(m < bound for _, m in ties), ties


def peak_margin2d(P, La, Le, wrap, i):
    """Relative margin of a 2-D peak (flat index i of an Le x La spectrum) over its neighbours."""
    P = np.asarray(P, np.float64).reshape(Le, La)
    l, k = divmod(int(i), La)
    nb = []
    for dl in (-1, 0, 1):
        for dk in (-1, 0, 1):
            if (dl or dk) and 0 <= l + dl < Le and (wrap or 0 <= k + dk < La):
                nb.append(P[l + dl, (k + dk) % La])
    return float((P[l, k] - max(nb)) / P[l, k]) if nb else 0.0


def compare_peaks2d(idx_gpu, idx_ref, P_ref, La, Le, wrap, bound):
    """2-D counterpart of compare_peaks: the flat index sets agree, or every disagreement is a tie
    within `bound` (margin of the oracle's point over its neighbours, or of the GPU's pick)."""
    a, b = list(idx_gpu), list(idx_ref)
    if a == b:
        return True, []
    diff = sorted(set(a) ^ set(b))
    ties = [(k, peak_margin2d(P_ref, La, Le, wrap, k)) for k in diff]
    return all(abs(m) < bound for _, m in ties), ties

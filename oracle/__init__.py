"""FP64 CPU oracle for noise-subspace DOA estimation (PHD, MUSIC, EV, MN).

TEST INFRASTRUCTURE, NOT PRODUCT CODE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. It shares no code with the CUDA
library in ``paper_2007_14135_gb300``; the two are written independently from the paper
(Eray & Temizel, arXiv 2007.14135).

The arithmetic lives in ``doa_oracle.c`` (plain C99, FP64, no FMA contraction). This module
compiles it with gcc on first use and exposes NumPy-friendly wrappers:

  covariance  -- Sec. 3.1 Eq. 3, Table 2 Step-1
  eigh        -- Table 2 Step-2 (cyclic Jacobi, eigenvalues descending)
  weighting   -- Table 3 Steps 3-4, explicit M x M matrix C
  scan        -- Table 2 Step-5 with the steering vector of Eq. 2 (half-wavelength ULA)
  peaks       -- Table 2 Step-6
  solve       -- Steps 1-6 for one snapshot matrix and one algorithm
  scan_geometry / peaks2d / solve_geometry
              -- Steps 5-6 (and 1-6) for an arbitrary array geometry on an azimuth x elevation grid,
                 steering vector of Eq. 2 as printed (Sec. 4.2's circular array)
  refine_peak / refine_peak2d
              -- sub-grid refinement of a picked peak: the local minimiser of a^H C a next to it
  model_order -- MDL / AIC source-count estimates from the eigenvalues (Wax & Kailath)
  svd_data    -- Step-2 as an SVD of the snapshot matrix X itself (one-sided Jacobi on its rows):
                 the eigenpairs of R = X X^H / N without forming R
  root_polynomial / root_music
              -- the ULA scan's denominator as a polynomial on the unit circle and its roots
                 (numpy.roots as the root finder)

The MLP oracle used for the learned proposal lives in ``oracle/mlp.py`` (NumPy, FP64).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

PHD, MUSIC, EV, MN = 0, 1, 2, 3
ALG_NAMES = {PHD: "PHD", MUSIC: "MUSIC", EV: "EV", MN: "MN"}

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "doa_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile doa_oracle.c into liboracle.so with gcc (plain -O2, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            d, i, p = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
            lib.oracle_covariance.argtypes = [p, i, i, i, p]
            lib.oracle_covariance.restype = None
            lib.oracle_eigh.argtypes = [p, i, d, i, p, p]
            lib.oracle_eigh.restype = i
            lib.oracle_weighting.argtypes = [p, p, i, i, i, p]
            lib.oracle_weighting.restype = i
            lib.oracle_scan.argtypes = [p, i, d, d, i, p, p]
            lib.oracle_scan.restype = None
            lib.oracle_peaks.argtypes = [p, i, i, p, p]
            lib.oracle_peaks.restype = i
            lib.oracle_solve.argtypes = [p, i, i, i, i, i, d, d, i, p, p, p, p, p]
            lib.oracle_solve.restype = i
            lib.oracle_scan_geometry.argtypes = [p, i, p, d, d, i, d, d, i, p]
            lib.oracle_scan_geometry.restype = None
            lib.oracle_peaks2d.argtypes = [p, i, i, i, i, p, p]
            lib.oracle_peaks2d.restype = i
            lib.oracle_refine_peak.argtypes = [p, i, d, d, i, p]
            lib.oracle_refine_peak.restype = d
            lib.oracle_refine_peak2d.argtypes = [p, i, p, d, d, i, d, d, i, p, p]
            lib.oracle_refine_peak2d.restype = None
            lib.oracle_model_order.argtypes = [p, i, i, p, p, p, p]
            lib.oracle_model_order.restype = None
            lib.oracle_svd_data.argtypes = [p, i, i, i, d, i, p, p]
            lib.oracle_svd_data.restype = i
            _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _as_c64_rows(X: np.ndarray) -> np.ndarray:
    X = np.ascontiguousarray(X, dtype=np.complex64)
    assert X.ndim == 2
    return X


def covariance(X: np.ndarray) -> np.ndarray:
    """R = X X^H / N (Eq. 3) for complex64 X of shape (M, N); returns complex128 (M, M)."""
    X = _as_c64_rows(X)
    M, N = X.shape
    R = np.empty((M, M), dtype=np.complex128)
    _load().oracle_covariance(_ptr(X), M, N, N, _ptr(R))
    return R


def eigh(R: np.ndarray, tol: float = 1e-15, max_sweeps: int = 100):
    """Cyclic Jacobi eigendecomposition. Returns (evals desc, V with eigenvectors as columns, sweeps).

    sweeps < 0 means the sweep cap was reached (-4).
    """
    R = np.ascontiguousarray(R, dtype=np.complex128)
    M = R.shape[0]
    ev = np.empty(M, dtype=np.float64)
    Vt = np.empty((M, M), dtype=np.complex128)  # row i = eigenvector i (column-major V)
    sweeps = _load().oracle_eigh(_ptr(R), M, tol, max_sweeps, _ptr(ev), _ptr(Vt))
    return ev, Vt.T.copy(), sweeps


def weighting(evals: np.ndarray, V: np.ndarray, D: int, alg: int):
    """Explicit weighting matrix C of Table 3. Returns (C, status); status 5 = rank failure."""
    evals = np.ascontiguousarray(evals, dtype=np.float64)
    M = evals.shape[0]
    Vt = np.ascontiguousarray(np.asarray(V, dtype=np.complex128).T)
    C = np.empty((M, M), dtype=np.complex128)
    st = _load().oracle_weighting(_ptr(evals), _ptr(Vt), M, D, alg, _ptr(C))
    return C, st


def grid_angles(lo: float, step: float, L: int) -> np.ndarray:
    """theta_k = lo + k*step (rounded product, then rounded sum), in degrees."""
    k = np.arange(L, dtype=np.float64)
    return lo + k * step


def scan(C: np.ndarray, lo: float, step: float, L: int):
    """P_k = 1 / (a_k^H C a_k) over the grid. Returns (P float64[L], max relative imaginary part)."""
    C = np.ascontiguousarray(C, dtype=np.complex128)
    M = C.shape[0]
    P = np.empty(L, dtype=np.float64)
    rel = ctypes.c_double(0.0)
    _load().oracle_scan(_ptr(C), M, float(lo), float(step), int(L), _ptr(P), ctypes.byref(rel))
    return P, rel.value


def peaks(P: np.ndarray, D: int):
    """Step-6 peak finding and selection. Returns (idx int32[count], val float64[count])."""
    P = np.ascontiguousarray(P, dtype=np.float64)
    idx = np.empty(max(D, 1), dtype=np.int32)
    val = np.empty(max(D, 1), dtype=np.float64)
    n = _load().oracle_peaks(_ptr(P), P.shape[0], D, _ptr(idx), _ptr(val))
    return idx[:n].copy(), val[:n].copy()


def solve(X: np.ndarray, D: int, alg: int, lo: float, step: float, L: int):
    """Steps 1-6 for one snapshot matrix. Returns dict(P, evals, C, idx, val, status)."""
    X = _as_c64_rows(X)
    M, N = X.shape
    P = np.empty(L, dtype=np.float64)
    ev = np.empty(M, dtype=np.float64)
    C = np.empty((M, M), dtype=np.complex128)
    idx = np.empty(max(D, 1), dtype=np.int32)
    val = np.empty(max(D, 1), dtype=np.float64)
    r = _load().oracle_solve(_ptr(X), M, N, N, D, alg, float(lo), float(step), int(L),
                             _ptr(P), _ptr(ev), _ptr(C), _ptr(idx), _ptr(val))
    status = -r if r < 0 else 0
    n = r if r >= 0 else 0
    return dict(P=P, evals=ev, C=C, idx=idx[:n].copy(), val=val[:n].copy(), status=status)


def uca_positions(M: int, radius_wl: float) -> np.ndarray:
    """Element positions (x, y, z) in wavelengths of an M-element uniform circular array of the
    given radius in the z = 0 plane, element m at angle 2 pi m / M from the +y axis towards +x
    (so that its azimuth matches the theta of Eq. 2). Returns float64 (M, 3)."""
    ang = 2.0 * np.pi * np.arange(M, dtype=np.float64) / M
    pos = np.zeros((M, 3), dtype=np.float64)
    pos[:, 0] = radius_wl * np.sin(ang)
    pos[:, 1] = radius_wl * np.cos(ang)
    return pos


def steering_geometry(pos: np.ndarray, theta_deg: float, phi_deg: float) -> np.ndarray:
    """Eq. 2 steering vector for positions in wavelengths (the same formula as the C scan, in
    NumPy, used to synthesise exact covariances in the tests)."""
    t, p = np.deg2rad(theta_deg), np.deg2rad(phi_deg)
    u = np.array([np.sin(t) * np.sin(p), np.cos(t) * np.sin(p), np.cos(p)])
    return np.exp(2j * np.pi * (np.asarray(pos, dtype=np.float64) @ u))


def scan_geometry(C: np.ndarray, pos: np.ndarray, az_lo: float, az_step: float, La: int,
                  el_lo: float, el_step: float, Le: int) -> np.ndarray:
    """P[l, k] = 1 / (a^H C a) at azimuth az_lo + k az_step, elevation el_lo + l el_step (degrees),
    steering of Eq. 2 for the element positions pos (M x 3, wavelengths). Returns float64 (Le, La)."""
    C = np.ascontiguousarray(C, dtype=np.complex128)
    M = C.shape[0]
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(M, 3)
    P = np.empty((Le, La), dtype=np.float64)
    _load().oracle_scan_geometry(_ptr(C), M, _ptr(pos), float(az_lo), float(az_step), int(La), float(el_lo),
                                 float(el_step), int(Le), _ptr(P))
    return P


def peaks2d(P: np.ndarray, D: int, wrap_az: bool):
    """Strict 8-neighbour maxima of an (Le, La) spectrum (azimuth wraps when wrap_az), the D largest
    (ties: lower flat index), returned as flat indices l*La + k in ascending order with values."""
    P = np.ascontiguousarray(P, dtype=np.float64)
    Le, La = P.shape
    idx = np.empty(max(D, 1), dtype=np.int32)
    val = np.empty(max(D, 1), dtype=np.float64)
    n = _load().oracle_peaks2d(_ptr(P), La, Le, int(bool(wrap_az)), D, _ptr(idx), _ptr(val))
    return idx[:n].copy(), val[:n].copy()


def solve_geometry(X: np.ndarray, D: int, alg: int, pos: np.ndarray, az_lo: float, az_step: float, La: int,
                   el_lo: float, el_step: float, Le: int, wrap_az: bool):
    """Steps 1-6 on an azimuth x elevation grid for an arbitrary geometry. Returns dict(P, evals, C,
    idx, val, status) with P of shape (Le, La) and idx flat indices."""
    R = covariance(X)
    ev, V, sweeps = eigh(R)
    if sweeps < 0:
        return dict(P=None, evals=ev, C=None, idx=np.empty(0, np.int32), val=np.empty(0), status=4)
    C, st = weighting(ev, V, D, alg)
    if st != 0:
        return dict(P=None, evals=ev, C=C, idx=np.empty(0, np.int32), val=np.empty(0), status=st)
    P = scan_geometry(C, pos, az_lo, az_step, La, el_lo, el_step, Le)
    idx, val = peaks2d(P, D, wrap_az)
    return dict(P=P, evals=ev, C=C, idx=idx, val=val, status=0)


def refine_peak(C: np.ndarray, lo: float, step: float, k: int):
    """Local minimiser (degrees) of a^H C a in the bracket around grid peak k of the ULA scan
    (bracketed Newton). Returns (theta, steps)."""
    C = np.ascontiguousarray(C, dtype=np.complex128)
    it = ctypes.c_int(0)
    th = _load().oracle_refine_peak(_ptr(C), C.shape[0], float(lo), float(step), int(k), ctypes.byref(it))
    return th, it.value


def refine_peak2d(C: np.ndarray, pos: np.ndarray, az_lo: float, az_step: float, La: int, el_lo: float,
                  el_step: float, flat: int):
    """Local minimiser (azimuth, elevation degrees) of a^H C a in the box around the 2-D grid peak
    with flat index l*La + k (damped Newton). Returns ((theta, phi), steps)."""
    C = np.ascontiguousarray(C, dtype=np.complex128)
    M = C.shape[0]
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(M, 3)
    out = np.zeros(2, dtype=np.float64)
    it = ctypes.c_int(0)
    _load().oracle_refine_peak2d(_ptr(C), M, _ptr(pos), float(az_lo), float(az_step), int(La), float(el_lo),
                                 float(el_step), int(flat), _ptr(out), ctypes.byref(it))
    return (float(out[0]), float(out[1])), it.value


def model_order(evals: np.ndarray, N: int):
    """MDL and AIC estimates of the number of sources from descending eigenvalues and the snapshot
    count. Returns (mdl, aic, mdl_values, aic_values)."""
    ev = np.ascontiguousarray(evals, dtype=np.float64)
    M = ev.shape[0]
    mv = np.empty(M)
    av = np.empty(M)
    m, a = ctypes.c_int(0), ctypes.c_int(0)
    _load().oracle_model_order(_ptr(ev), M, int(N), ctypes.byref(m), ctypes.byref(a), _ptr(mv), _ptr(av))
    return m.value, a.value, mv, av


def root_polynomial(C: np.ndarray) -> np.ndarray:
    """Coefficients of the root form of the ULA scan's denominator: on |z| = 1, with z = e^{j pi sin
    theta}, a(theta)^H C a(theta) = sum_l c_l z^l, c_l = sum over the l-th diagonal (j - i = l) of C.
    Returned highest power first (numpy.roots order) for z^{M-1} D(z), degree 2M-2."""
    C = np.asarray(C, dtype=np.complex128)
    M = C.shape[0]
    c = np.zeros(2 * M - 1, dtype=np.complex128)          # c[l + M - 1] = c_l
    for i in range(M):
        for j in range(M):
            c[j - i + M - 1] += C[i, j]
    return c[::-1].copy()


def root_music(C: np.ndarray, d: int):
    """Root-MUSIC on the ULA: the roots of z^{M-1} D(z) (numpy.roots: companion-matrix eigenvalues)
    come in pairs z, 1/conj(z); the d roots with |z| <= 1 closest to the unit circle give the
    angles theta = asin(arg(z) / pi) (degrees, ascending). Returns (angles, selected roots)."""
    roots = np.roots(root_polynomial(C))
    inside = roots[np.abs(roots) <= 1.0]
    order = np.argsort(-np.abs(inside), kind="stable")
    pick = inside[order[:d]]
    ang = np.degrees(np.arcsin(np.clip(np.angle(pick) / np.pi, -1.0, 1.0)))
    o = np.argsort(ang)
    return ang[o], pick[o]


def svd_data(X: np.ndarray, tol: float = 1e-15, max_sweeps: int = 100):
    """One-sided Jacobi SVD of the M x N snapshot matrix X (complex64 or complex128; complex64 is
    promoted exactly). Returns (evals, U, sweeps) in the form of eigh: the eigenvalues S_k^2 / N of
    R = X X^H / N descending, U with the left singular vectors as columns, and the sweep count
    (negative: the sweep cap was reached)."""
    X = np.ascontiguousarray(X, dtype=np.complex128)
    assert X.ndim == 2
    M, N = X.shape
    ev = np.empty(M, dtype=np.float64)
    Ut = np.empty((M, M), dtype=np.complex128)   # row i = singular vector i (column-major U)
    sweeps = _load().oracle_svd_data(_ptr(X), M, N, N, tol, max_sweeps, _ptr(ev), _ptr(Ut))
    return ev, Ut.T.copy(), sweeps

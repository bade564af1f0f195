"""Thin Python binding of libdoa.so (C ABI declared in include/doa.h).

Argument marshalling only: every step of the method runs in the library's CUDA kernels.
PyTorch supplies device memory and streams. The library must have been built
(``paper_2007_14135_gb300.build.build()``); importing this module without it raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdoa.so")

PHD, MUSIC, EV, MN = 0, 1, 2, 3
FP32, BF16, BF16X3, FP16X3 = 0, 1, 2, 3
EIG_DOUBLE_FLOAT, EIG_FP64 = 0, 1
FLAG_POLISH_PEAKS = 1
FLAG_COV_CUDA_CORE = 2
OK, EINVAL, ENOMEM, ECUDA, ENOCONV, ERANK, ENONFINITE, ETIMEOUT = range(8)
NOALLOC_SCRATCH_BYTES = 4 << 20
BATCH_STAGES = 5
STAGE_NAMES = ("phase_tables", "covariance", "eig_noise_subspace", "scan", "peaks")

# every symbol include/doa.h declares
EXPORTS = ("doa_status_str", "doa_covariance", "doa_covariance_noalloc", "doa_noise_subspace", "doa_scan",
           "doa_peaks", "doa_batch_plan_bytes", "doa_batch_plan", "doa_solve_batch", "doa_mlp_workspace_bytes",
           "doa_mlp_refresh", "doa_mlp_forward", "doa_mlp_backward", "doa_mlp_adam", "doa_synth_ula",
           "doa_proposal_windows", "doa_scan_windows", "doa_scan_slice", "doa_slice_peaks", "doa_merge_slices", "doa_probe_fma",
           "doa_scan_geometry", "doa_scan_geometry_ws_bytes", "doa_peaks2d", "doa_refine_peaks",
           "doa_refine_peaks2d", "doa_model_order", "doa_root_music", "doa_proposal_judge", "doa_svd_data",
           "doa_svd_data_ws_bytes", "doa_noise_subspace_prec")
SLICE_MAXD = 64


class DoaError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {status_str(status)} ({status})")
        self.status = status


class Grid(ctypes.Structure):
    _fields_ = [("lo_deg", ctypes.c_double), ("step_deg", ctypes.c_double),
                ("L", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class Geometry(ctypes.Structure):
    """doa_geometry: element positions (device, M x 3 FP64, wavelengths) and the elevation rows of a
    2-D azimuth x elevation scan; pos = NULL means the 1-D ULA scan."""
    _fields_ = [("pos", ctypes.c_void_p), ("el_lo_deg", ctypes.c_double), ("el_step_deg", ctypes.c_double),
                ("Le", ctypes.c_int32), ("wrap_az", ctypes.c_int32)]


class Problem(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("P", ctypes.c_void_p), ("peak_idx", ctypes.c_void_p),
                ("peak_val", ctypes.c_void_p), ("peak_count", ctypes.c_void_p),
                ("evals", ctypes.c_void_p), ("grid", Grid), ("M", ctypes.c_int32),
                ("N", ctypes.c_int32), ("ldx", ctypes.c_int32), ("d", ctypes.c_int32),
                ("alg_mask", ctypes.c_uint32), ("prec", ctypes.c_int32), ("features", ctypes.c_void_p),
                ("B_out", ctypes.c_void_p), ("eig_prec", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("geom", Geometry), ("peak_angle", ctypes.c_void_p), ("order_est", ctypes.c_void_p),
                ("root_angle", ctypes.c_void_p)]


class SliceSummary(ctypes.Structure):
    """doa_slice_summary: decided peaks of one grid slice plus what the merge needs at its edges."""
    _fields_ = [("count", ctypes.c_int32), ("open_idx", ctypes.c_int32), ("open_val", ctypes.c_float),
                ("first_val", ctypes.c_float), ("first_run_to_end", ctypes.c_int32),
                ("first_next_val", ctypes.c_float), ("idx", ctypes.c_int32 * 64), ("val", ctypes.c_float * 64)]


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    if not os.path.exists(path):
        raise RuntimeError(f"libdoa.so is missing at {path}: run paper_2007_14135_gb300.build.build()")
    lib = ctypes.CDLL(path)
    vp, i, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
    lib.doa_status_str.argtypes = [i]
    lib.doa_status_str.restype = ctypes.c_char_p
    lib.doa_covariance.argtypes = [vp, i, i, i, vp, vp, i, vp]
    lib.doa_covariance_noalloc.argtypes = [vp, i, i, i, vp, vp, vp]
    lib.doa_noise_subspace.argtypes = [vp, i, i, i, vp, vp, vp, vp, vp]
    lib.doa_noise_subspace_prec.argtypes = [vp, i, i, i, i, vp, vp, vp, vp, vp]
    lib.doa_scan.argtypes = [vp, i, i, Grid, i, vp, vp]
    lib.doa_peaks.argtypes = [vp, i, i, vp, vp, vp, vp]
    lib.doa_batch_plan_bytes.argtypes = [ctypes.POINTER(Problem), i]
    lib.doa_batch_plan_bytes.restype = sz
    lib.doa_batch_plan.argtypes = [ctypes.POINTER(Problem), i, vp, vp, sz, ctypes.POINTER(sz),
                                   ctypes.POINTER(ctypes.c_int)]
    lib.doa_solve_batch.argtypes = [vp, vp, vp, sz, vp, vp, vp]
    lib.doa_scan_slice.argtypes = [vp, i, i, Grid, i, i, vp, vp]
    lib.doa_slice_peaks.argtypes = [vp, i, i, i, i, i, vp, vp]
    lib.doa_merge_slices.argtypes = [vp, i, i, vp, vp, vp]
    lib.doa_probe_fma.argtypes = [i, i, i, vp, ctypes.POINTER(ctypes.c_double), vp]
    lib.doa_scan_geometry.argtypes = [vp, i, i, Grid, Geometry, vp, vp, sz, vp]
    lib.doa_scan_geometry_ws_bytes.argtypes = [i, i]
    lib.doa_scan_geometry_ws_bytes.restype = sz
    lib.doa_peaks2d.argtypes = [vp, i, i, i, i, vp, vp, vp, vp]
    lib.doa_refine_peaks.argtypes = [vp, i, i, Grid, vp, vp, i, vp, vp]
    lib.doa_model_order.argtypes = [vp, i, i, vp, vp, vp]
    lib.doa_root_music.argtypes = [vp, i, i, i, vp, vp, vp]
    lib.doa_refine_peaks2d.argtypes = [vp, i, i, Grid, Geometry, vp, vp, i, vp, vp]
    lib.doa_svd_data_ws_bytes.argtypes = [i, i]
    lib.doa_svd_data_ws_bytes.restype = sz
    lib.doa_svd_data.argtypes = [vp, i, i, i, i, ctypes.c_double, i, vp, vp, vp, vp, sz, vp]
    for name in ("doa_covariance", "doa_covariance_noalloc", "doa_noise_subspace", "doa_scan", "doa_peaks",
                 "doa_batch_plan", "doa_solve_batch", "doa_scan_slice", "doa_slice_peaks", "doa_merge_slices", "doa_probe_fma",
                 "doa_scan_geometry", "doa_peaks2d", "doa_refine_peaks", "doa_refine_peaks2d", "doa_model_order",
                 "doa_root_music", "doa_proposal_judge", "doa_svd_data", "doa_noise_subspace_prec"):
        getattr(lib, name).restype = i
    return lib


_lib: Optional[ctypes.CDLL] = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        _lib = load_library()
    return _lib


def status_str(status: int) -> str:
    return lib().doa_status_str(int(status)).decode()


def _check(status: int, where: str) -> None:
    if status != OK:
        raise DoaError(status, where)


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def _dev(t: Optional[torch.Tensor]) -> Optional[int]:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("device tensor expected")
    return t.data_ptr()


def grid(lo: float, step: float, L: int) -> Grid:
    return Grid(float(lo), float(step), int(L), 0)


def geometry(pos: torch.Tensor, el_lo: float, el_step: float, Le: int, wrap_az: bool) -> Geometry:
    """doa_geometry for device positions pos (float64, (M, 3), contiguous; must outlive its use)."""
    assert pos.dtype == torch.float64 and pos.is_contiguous() and pos.dim() == 2 and pos.shape[1] == 3
    return Geometry(_dev(pos), float(el_lo), float(el_step), int(Le), 1 if wrap_az else 0)


# ------------------------------------------------------------------------------------ stages
def doa_covariance(X: torch.Tensor, R: Optional[torch.Tensor] = None, R64: Optional[torch.Tensor] = None,
                   prec: int = FP32, stream=None) -> None:
    """R = X X^H / N. X: complex64 (M, N) with unit column stride (row stride = ldx)."""
    assert X.dtype == torch.complex64 and X.dim() == 2 and X.stride(1) == 1
    M, N = X.shape
    _check(lib().doa_covariance(_dev(X), M, N, X.stride(0), _dev(R), _dev(R64), prec, _stream(stream)),
           "doa_covariance")


def doa_covariance_noalloc(X: torch.Tensor, R: Optional[torch.Tensor] = None, R64: Optional[torch.Tensor] = None,
                           stream=None) -> None:
    """Same as doa_covariance, but the library allocates nothing and takes no workspace: the
    chunk sums live in a fixed library-owned device array (DOA_NOALLOC_SCRATCH_BYTES), for
    callers that cannot allocate while running. Calls that overlap on one GPU race on it."""
    assert X.dtype == torch.complex64 and X.dim() == 2 and X.stride(1) == 1
    M, N = X.shape
    _check(lib().doa_covariance_noalloc(_dev(X), M, N, X.stride(0), _dev(R), _dev(R64), _stream(stream)),
           "doa_covariance_noalloc")


def doa_noise_subspace(R64: torch.Tensor, d: int, alg: int, B: torch.Tensor, info: torch.Tensor,
                       evals: Optional[torch.Tensor] = None, K_out: Optional[torch.Tensor] = None,
                       stream=None) -> None:
    """Jacobi eig of R64 (complex128 (M, M)) and the factor B (complex128, M*M capacity)."""
    M = R64.shape[0]
    assert R64.dtype == torch.complex128 and B.dtype == torch.complex128 and B.numel() >= M * M
    _check(lib().doa_noise_subspace(_dev(R64), M, d, alg, _dev(evals), _dev(B), _dev(K_out), _dev(info),
                                    _stream(stream)), "doa_noise_subspace")


def doa_noise_subspace_prec(R64: torch.Tensor, d: int, alg: int, eig_prec: int, B: torch.Tensor, info: torch.Tensor,
                            evals: Optional[torch.Tensor] = None, K_out: Optional[torch.Tensor] = None,
                            stream=None) -> None:
    """doa_noise_subspace with the Jacobi's arithmetic chosen (EIG_DOUBLE_FLOAT or EIG_FP64)."""
    M = R64.shape[0]
    assert R64.dtype == torch.complex128 and B.dtype == torch.complex128 and B.numel() >= M * M
    _check(lib().doa_noise_subspace_prec(_dev(R64), M, d, alg, eig_prec, _dev(evals), _dev(B), _dev(K_out),
                                         _dev(info), _stream(stream)), "doa_noise_subspace_prec")


def doa_scan(B: torch.Tensor, M: int, K: int, g: Grid, P: torch.Tensor, prec: int = FP32, stream=None) -> None:
    """P_k = 1/||B^H a(theta_k)||^2 for the grid. B: complex128, column-major (ld M)."""
    assert B.dtype == torch.complex128 and P.dtype == torch.float32 and P.numel() >= g.L
    _check(lib().doa_scan(_dev(B), M, K, g, prec, _dev(P), _stream(stream)), "doa_scan")


def doa_scan_slice(B: torch.Tensor, M: int, K: int, g: Grid, k0: int, n: int, P: torch.Tensor, stream=None) -> None:
    """The global grid points k0 .. k0+n-1 of doa_scan (FP32 path) into P[0..n)."""
    assert B.dtype == torch.complex128 and P.dtype == torch.float32 and P.numel() >= n
    _check(lib().doa_scan_slice(_dev(B), M, K, g, k0, n, _dev(P), _stream(stream)), "doa_scan_slice")


def doa_slice_peaks(Pbuf: torch.Tensor, b0: int, k0: int, k1: int, L: int, d: int, out: torch.Tensor,
                    stream=None) -> None:
    """Peak summary of the slice [k0, k1); Pbuf holds global points b0 .. min(k1+1, L)-1 and out is
    a device byte tensor of ctypes.sizeof(SliceSummary) bytes."""
    assert Pbuf.dtype == torch.float32 and out.numel() * out.element_size() >= ctypes.sizeof(SliceSummary)
    _check(lib().doa_slice_peaks(_dev(Pbuf), b0, k0, k1, L, d, _dev(out), _stream(stream)), "doa_slice_peaks")


def slice_summary_from_bytes(raw: bytes) -> SliceSummary:
    return SliceSummary.from_buffer_copy(raw[:ctypes.sizeof(SliceSummary)])


def doa_merge_slices(sums: Sequence[SliceSummary], d: int):
    """Host merge of per-slice summaries (slice order) -> (indices, values), as doa_peaks."""
    arr = (SliceSummary * len(sums))(*sums)
    idx = (ctypes.c_int32 * max(d, 1))()
    val = (ctypes.c_float * max(d, 1))()
    cnt = ctypes.c_int32(0)
    _check(lib().doa_merge_slices(ctypes.cast(arr, ctypes.c_void_p), len(sums), d, ctypes.cast(idx, ctypes.c_void_p),
                                  ctypes.cast(val, ctypes.c_void_p), ctypes.cast(ctypes.pointer(cnt), ctypes.c_void_p)),
           "doa_merge_slices")
    n = cnt.value
    return np.array(idx[:n], dtype=np.int32), np.array(val[:n], dtype=np.float32)


def probe_fma_tflops(fp64, device: str = "cuda", iters: int = 1 << 14, reps: int = 5) -> float:
    """Measured FMA rate (TFLOP/s, best of `reps`) of FP32 (False / 0), FP64 (True / 1) or paired
    FP32 (2: fma.rn.f32x2) chains on every SM."""
    mode = int(fp64)
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    blocks = sms * 8
    out = torch.empty(blocks * 256, dtype=torch.float64 if mode == 1 else torch.float32, device=device)
    flops = ctypes.c_double(0.0)
    best = 0.0
    for _ in range(reps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        _check(lib().doa_probe_fma(mode, blocks, iters, _dev(out), ctypes.byref(flops), _stream(None)),
               "doa_probe_fma")
        e1.record()
        torch.cuda.synchronize()
        best = max(best, flops.value / (e0.elapsed_time(e1) / 1e3) / 1e12)
    return best


def doa_peaks(P: torch.Tensor, d: int, idx: torch.Tensor, val: torch.Tensor, count: torch.Tensor,
              L: Optional[int] = None, stream=None) -> None:
    L = P.numel() if L is None else L
    _check(lib().doa_peaks(_dev(P), L, d, _dev(idx), _dev(val), _dev(count), _stream(stream)), "doa_peaks")


def doa_scan_geometry(B: torch.Tensor, M: int, K: int, az: Grid, geom: Geometry, P: torch.Tensor,
                      ws: Optional[torch.Tensor] = None, stream=None) -> None:
    """2-D scan P[l * La + k] over azimuth az (columns) and the rows of geom (Eq. 2 as printed).
    ws: device scratch for the grid's sin / cos tables (allocated here when None)."""
    need = lib().doa_scan_geometry_ws_bytes(az.L, geom.Le)
    if ws is None:
        ws = torch.empty(max(need, 16), dtype=torch.uint8, device=B.device)
    _check(lib().doa_scan_geometry(_dev(B), M, K, az, geom, _dev(P), _dev(ws), ws.numel() * ws.element_size(),
                                   _stream(stream)), "doa_scan_geometry")


def doa_root_music(B: torch.Tensor, M: int, K: int, d: int, theta: torch.Tensor, info: torch.Tensor,
                   stream=None) -> None:
    """Root form of the ULA scan: d angles (degrees, ascending) from the polynomial's roots."""
    assert theta.dtype == torch.float64 and theta.numel() >= d
    _check(lib().doa_root_music(_dev(B), M, K, d, _dev(theta), _dev(info), _stream(stream)), "doa_root_music")


def doa_model_order(evals: torch.Tensor, N: int, out: torch.Tensor, stream=None) -> None:
    """MDL and AIC source-count estimates (out: 2 int32 on the device) from descending eigenvalues."""
    _check(lib().doa_model_order(_dev(evals), evals.numel(), N, _dev(out), out.data_ptr() + 4, _stream(stream)),
           "doa_model_order")


def svd_data_ws_bytes(M: int, N: int) -> int:
    return int(lib().doa_svd_data_ws_bytes(M, N))


def doa_svd_data(X: torch.Tensor, evals: torch.Tensor, U: torch.Tensor, info: torch.Tensor, ws: torch.Tensor = None,
                 tol: float = 1e-15, max_sweeps: int = 60, stream=None) -> torch.Tensor:
    """Step-2 as a one-sided Jacobi SVD of X (M x N complex64 or complex128 on the device, unit
    inner stride): evals (M float64, descending), U (M x M complex128; its transpose is the
    column-major array the call writes, so U[k] is singular vector k), info (1 int32: sweeps or
    -ENOCONV). ws: None (allocated here) or a uint8 device buffer. Returns ws."""
    assert X.dim() == 2 and X.stride(1) == 1 and X.dtype in (torch.complex64, torch.complex128)
    M, N = X.shape
    assert evals.dtype == torch.float64 and U.dtype == torch.complex128 and info.dtype == torch.int32
    need = svd_data_ws_bytes(M, N)
    if ws is None:
        ws = torch.empty(max(need, 256), dtype=torch.uint8, device=X.device)
    _check(lib().doa_svd_data(_dev(X), 1 if X.dtype == torch.complex128 else 0, M, N, X.stride(0), tol, max_sweeps,
                              _dev(evals), _dev(U), _dev(info), _dev(ws), ws.numel(), _stream(stream)),
           "doa_svd_data")
    return ws


def doa_refine_peaks(B: torch.Tensor, M: int, K: int, g: Grid, idx: torch.Tensor, count: torch.Tensor,
                     theta: torch.Tensor, stream=None) -> None:
    """Sub-grid refinement (FP64 bracketed Newton) of the peaks idx[:count] of a ULA scan."""
    assert theta.dtype == torch.float64
    _check(lib().doa_refine_peaks(_dev(B), M, K, g, _dev(idx), _dev(count), min(idx.numel(), theta.numel()),
                                  _dev(theta), _stream(stream)), "doa_refine_peaks")


def doa_refine_peaks2d(B: torch.Tensor, M: int, K: int, az: Grid, geom: Geometry, idx: torch.Tensor,
                       count: torch.Tensor, out: torch.Tensor, stream=None) -> None:
    """Sub-grid refinement (FP64 damped Newton) of 2-D peaks: out holds (azimuth, elevation) pairs."""
    assert out.dtype == torch.float64
    _check(lib().doa_refine_peaks2d(_dev(B), M, K, az, geom, _dev(idx), _dev(count), min(idx.numel(), out.numel() // 2),
                                    _dev(out), _stream(stream)), "doa_refine_peaks2d")


def doa_peaks2d(P: torch.Tensor, La: int, Le: int, wrap_az: bool, d: int, idx: torch.Tensor, val: torch.Tensor,
                count: torch.Tensor, stream=None) -> None:
    _check(lib().doa_peaks2d(_dev(P), La, Le, 1 if wrap_az else 0, d, _dev(idx), _dev(val), _dev(count),
                             _stream(stream)), "doa_peaks2d")


# ------------------------------------------------------------------------------------ batch
def make_problem(X: torch.Tensor, d: int, alg_mask: int, g: Grid, P: torch.Tensor, peak_idx: torch.Tensor,
                 peak_val: torch.Tensor, peak_count: torch.Tensor, evals: Optional[torch.Tensor] = None,
                 prec: int = FP32, features: Optional[torch.Tensor] = None,
                 B_out: Optional[torch.Tensor] = None, eig_prec: int = 0, polish: bool = False,
                 geom: Optional[Geometry] = None, peak_angle: Optional[torch.Tensor] = None,
                 order_est: Optional[torch.Tensor] = None, root_angle: Optional[torch.Tensor] = None,
                 cov_cuda_core: bool = False) -> Problem:
    """Descriptor of one problem; the tensors must outlive every solve that uses it. With geom the
    problem is a 2-D scan: g is the azimuth grid, P holds nalg x (Le x La) floats. cov_cuda_core
    selects the compensated CUDA-core covariance instead of the tensor-core one (M <= 16)."""
    assert X.dtype == torch.complex64 and X.dim() == 2 and X.stride(1) == 1
    M, N = X.shape
    return Problem(_dev(X), _dev(P), _dev(peak_idx), _dev(peak_val), _dev(peak_count), _dev(evals), g,
                   M, N, X.stride(0), d, alg_mask, prec, _dev(features), _dev(B_out), eig_prec,
                   (FLAG_POLISH_PEAKS if polish else 0) | (FLAG_COV_CUDA_CORE if cov_cuda_core else 0), geom if geom is not None else Geometry(None, 0.0, 0.0, 0, 0),
                   _dev(peak_angle), _dev(order_est), _dev(root_angle))


class Tuning(ctypes.Structure):
    """doa_tuning: per-M-bucket launch shapes (0 = default)."""
    _fields_ = [("scan_pt", ctypes.c_int32 * 4), ("eig_mats", ctypes.c_int32 * 4), ("scan_group", ctypes.c_int32 * 4)]


class BatchPlan:
    """Host plan bytes, their device copy, and the workspace size (doa_batch_plan).

    scan_pt: None or 4 ints (grid points per scan thread for M <= 8, 16, 32, 64; 0 = default).
    eig_mats: None or 4 ints (matrices per Jacobi warp per bucket; 0 = default).
    scan_group: None or 4 ints (problems sharing a grid scanned together per bucket; 1 = each alone;
    0 = default)."""

    def __init__(self, problems: Sequence[Problem], device: str = "cuda", scan_pt: Optional[Sequence[int]] = None,
                 eig_mats: Optional[Sequence[int]] = None, scan_group: Optional[Sequence[int]] = None):
        arr = (Problem * len(problems))(*problems)
        tun = None
        if scan_pt is not None or eig_mats is not None or scan_group is not None:
            tun = Tuning((ctypes.c_int32 * 4)(*[int(v) for v in (scan_pt or (0, 0, 0, 0))]),
                         (ctypes.c_int32 * 4)(*[int(v) for v in (eig_mats or (0, 0, 0, 0))]),
                         (ctypes.c_int32 * 4)(*[int(v) for v in (scan_group or (0, 0, 0, 0))]))
        tun_ptr = None if tun is None else ctypes.cast(ctypes.pointer(tun), ctypes.c_void_p)
        n = lib().doa_batch_plan_bytes(arr, len(problems))
        ws = ctypes.c_size_t(0)
        bad = ctypes.c_int(-1)
        if n == 0:
            st = lib().doa_batch_plan(arr, len(problems), tun_ptr, None, 0, ctypes.byref(ws), ctypes.byref(bad))
            raise DoaError(st if st else EINVAL, f"doa_batch_plan (problem {bad.value})")
        self.host = np.zeros(n, dtype=np.uint8)
        _check(lib().doa_batch_plan(arr, len(problems), tun_ptr, self.host.ctypes.data, n, ctypes.byref(ws),
                                    ctypes.byref(bad)), f"doa_batch_plan (problem {bad.value})")
        self.ws_bytes = int(ws.value)
        self.nprob = len(problems)
        hdr = self.host[:256].view(np.int32)
        self.scan_pt = [int(v) for v in hdr[self.header_index("scan_pt"):][:4]]
        self.eig_mats = [int(v) for v in hdr[self.header_index("eig_mats"):][:4]]
        self.scan_group = [int(v) for v in self.host[:1024].view(np.int32)[116:120]]
        self.dev = torch.from_numpy(self.host).to(device)
        self.problems = arr

    @staticmethod
    def header_index(field: str) -> int:
        """int32 index of a PlanHeader field (layout of csrc/doa_internal.cuh)."""
        order = {"magic": 0, "nprob": 1, "njobs": 2, "ngrids": 3, "ncov": 4, "nreduce": 5, "eig_count": 6,
                 "scan_jobs": 10, "scan_tiles": 14, "scan_pt": 22, "eig_mats": 58, "cov_first": 62, "tc_jobs": 67,
                 "npolish": 74, "geo_jobs": 76, "ngeo_grids": 96, "nrefine": 100, "nroots": 101,
                 "ngeo_steer": 104, "ncovtc": 108, "covtc_flag_off": 114}
        return order[field]

    def launches(self) -> int:
        """Kernels one doa_solve_batch of this plan launches."""
        h = self.host[:1024].view(np.int32)
        cf = [int(v) for v in h[62:67]]                       # cov_first: classes MB = 2, 3, 4, other
        cov = sum(2 for c in range(3) if cf[c + 1] > cf[c]) + int(cf[4] > cf[3]) + int(h[5] > 0)
        eig_b = sum(int(c) > 0 for c in h[6:10])
        scan_b = sum(int(c) > 0 for c in h[10:14]) + int(h[67] > 0) + sum(int(c) > 0 for c in h[76:80])
        ngeo = sum(int(c) for c in h[76:80])
        peaks = int(ngeo < int(h[1])) + int(ngeo > 0) + (2 if int(h[74]) > 0 else 0)
        covtc = int(h[108] > 0) + int(h[109] > 0)
        covtc += int(covtc > 0)                                # the fixup kernel after them
        # grid-shared scan: a prep kernel and the scan kernel per M bucket that has groups
        shared = 2 * sum(int(u) > 0 for u in self.host[496:528].view(np.int64))
        shared += 2 * int(h[152] > 0)                          # tensor-core groups: prep + scan
        return (int(h[3] > 0) + int(h[96] > 0) + int(h[104] > 0) + cov + covtc + eig_b + scan_b + shared + peaks
                + int(h[100] > 0) + int(h[101] > 0))

    def covariance(self, ws: torch.Tensor, i: int) -> torch.Tensor:
        """Problem i's covariance R (M x M complex128) in the workspace after a solve (a view)."""
        off_prob = int(self.host[:512][120:128].view(np.int64)[0])
        rec = off_prob + i * (ctypes.sizeof(Problem) + 96)
        r64 = int(self.host[rec + ctypes.sizeof(Problem):rec + ctypes.sizeof(Problem) + 8].view(np.int64)[0])
        M = int(self.problems[i].M)
        return ws[r64:r64 + 16 * M * M].view(torch.complex128).view(M, M)

    def covtc_marks(self, ws: torch.Tensor) -> torch.Tensor:
        """The tensor-core covariance's per-problem marks from the workspace after a solve (0: done on
        the tensor cores; 1: a sample outside the scaling range; 2: a bounded wait ran out; marked
        problems were recomputed by the CUDA-core fixup)."""
        h = self.host[:512]
        n = int(h[432:440].view(np.int32).sum())
        off = int(h[456:464].view(np.int64)[0])
        return ws[off:off + 4 * n].view(torch.int32)


def doa_solve_batch(plan: BatchPlan, ws: torch.Tensor, status: torch.Tensor, stage_events=None,
                    stream=None) -> None:
    """Runs the plan. stage_events: None or DOA_BATCH_STAGES + 1 torch.cuda.Event (enable_timing)."""
    assert ws.numel() * ws.element_size() >= plan.ws_bytes and status.numel() >= plan.nprob
    ev = None
    if stage_events is not None:
        assert len(stage_events) == BATCH_STAGES + 1
        for e in stage_events:      # torch creates the CUDA event on its first record
            if not e.cuda_event:
                e.record(torch.cuda.current_stream() if stream is None else stream)
        ev = (ctypes.c_void_p * len(stage_events))(*[e.cuda_event for e in stage_events])
    _check(lib().doa_solve_batch(plan.host.ctypes.data, _dev(plan.dev), _dev(ws), plan.ws_bytes, _dev(status),
                                 ev, _stream(stream)), "doa_solve_batch")


def workspace(plan: BatchPlan, device: str = "cuda") -> torch.Tensor:
    """A device buffer of the plan's workspace size (256-byte aligned by the caching allocator)."""
    return torch.empty(max(plan.ws_bytes, 256), dtype=torch.uint8, device=device)


# ------------------------------------------------------------------------------------ network
MLP_DIMS = (272, 256, 256, 256, 181)


class MlpStruct(ctypes.Structure):
    _fields_ = [(name, ctypes.c_void_p * 4) for name in
                ("W", "b", "mW", "vW", "mb", "vb", "gW", "gb", "Wh", "WhT")]


def _bind_mlp(lib_):
    vp, i, sz, f = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t, ctypes.c_float
    lib_.doa_mlp_workspace_bytes.argtypes = [i]
    lib_.doa_mlp_workspace_bytes.restype = sz
    lib_.doa_mlp_refresh.argtypes = [ctypes.POINTER(MlpStruct), vp]
    lib_.doa_mlp_forward.argtypes = [ctypes.POINTER(MlpStruct), vp, i, vp, vp, vp, sz, vp]
    lib_.doa_mlp_backward.argtypes = [ctypes.POINTER(MlpStruct), vp, vp, i, vp, vp, sz, vp]
    lib_.doa_mlp_adam.argtypes = [ctypes.POINTER(MlpStruct), f, f, f, f, i, vp]
    for n in ("doa_mlp_refresh", "doa_mlp_forward", "doa_mlp_backward", "doa_mlp_adam"):
        getattr(lib_, n).restype = i


class Mlp:
    """Device buffers of the proposal network (doa_mlp) and thin wrappers of its entry points.

    Initial weights: He-uniform (bound sqrt(6 / fan_in)) from a seeded NumPy Philox generator,
    biases zero, Adam moments zero."""

    def __init__(self, seed: int = 0, device: str = "cuda", train: bool = True):
        _bind_mlp(lib())
        self.device = device
        rng = np.random.Generator(np.random.Philox(key=int(seed)))
        self.t = 0
        fields = ("W", "b", "mW", "vW", "mb", "vb", "gW", "gb", "Wh", "WhT")
        self.buf = {k: [] for k in fields}
        for l in range(4):
            fin, fout = MLP_DIMS[l], MLP_DIMS[l + 1]
            bound = np.sqrt(6.0 / fin)
            W = rng.uniform(-bound, bound, size=(fout, fin)).astype(np.float32)
            self.buf["W"].append(torch.from_numpy(W).to(device))
            self.buf["b"].append(torch.zeros(fout, dtype=torch.float32, device=device))
            for k, shape in (("mW", (fout, fin)), ("vW", (fout, fin)), ("gW", (fout, fin)),
                             ("mb", (fout,)), ("vb", (fout,)), ("gb", (fout,))):
                self.buf[k].append(torch.zeros(shape, dtype=torch.float32, device=device) if train else None)
            self.buf["Wh"].append(torch.zeros((fout, fin), dtype=torch.bfloat16, device=device))
            self.buf["WhT"].append(torch.zeros((fin, (fout + 7) // 8 * 8), dtype=torch.bfloat16, device=device))
        self.struct = MlpStruct()
        for k in fields:
            arr = getattr(self.struct, k)
            for l in range(4):
                t = self.buf[k][l]
                arr[l] = t.data_ptr() if t is not None else None
        self.refresh()

    def refresh(self, stream=None):
        _check(lib().doa_mlp_refresh(ctypes.byref(self.struct), _stream(stream)), "doa_mlp_refresh")

    def workspace(self, batch: int) -> torch.Tensor:
        n = lib().doa_mlp_workspace_bytes(batch)
        if n == 0:
            raise DoaError(EINVAL, "doa_mlp_workspace_bytes (batch must be a positive multiple of 8)")
        return torch.empty(n, dtype=torch.uint8, device=self.device)

    def forward(self, features: torch.Tensor, ws: torch.Tensor, probs=None, logits=None, stream=None):
        B = features.shape[0]
        _check(lib().doa_mlp_forward(ctypes.byref(self.struct), _dev(features), B, _dev(probs), _dev(logits),
                                     _dev(ws), ws.numel(), _stream(stream)), "doa_mlp_forward")

    def backward(self, features: torch.Tensor, labels: torch.Tensor, ws: torch.Tensor, loss=None, stream=None):
        B = features.shape[0]
        _check(lib().doa_mlp_backward(ctypes.byref(self.struct), _dev(features), _dev(labels), B, _dev(loss),
                                      _dev(ws), ws.numel(), _stream(stream)), "doa_mlp_backward")

    def adam(self, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8, stream=None):
        self.t += 1
        _check(lib().doa_mlp_adam(ctypes.byref(self.struct), lr, beta1, beta2, eps, self.t, _stream(stream)),
               "doa_mlp_adam")

    def params_numpy(self):
        return [(self.buf["W"][l].cpu().numpy().astype(np.float64), self.buf["b"][l].cpu().numpy().astype(np.float64))
                for l in range(4)]

    def save(self, path: str) -> None:
        """Checkpoint: magic, Adam step, then every FP32 buffer (W, b, moments) in layer order."""
        with open(path, "wb") as f:
            f.write(np.array([0x4D4C5031, self.t], dtype=np.int64).tobytes())
            for k in ("W", "b", "mW", "vW", "mb", "vb"):
                for l in range(4):
                    t = self.buf[k][l]
                    f.write((t if t is not None else torch.zeros(1)).detach().cpu().numpy().astype(np.float32).tobytes())

    def load(self, path: str) -> None:
        raw = open(path, "rb").read()
        head = np.frombuffer(raw[:16], dtype=np.int64)
        if head[0] != 0x4D4C5031:
            raise ValueError("not a network checkpoint")
        self.t = int(head[1])
        at = 16
        for k in ("W", "b", "mW", "vW", "mb", "vb"):
            for l in range(4):
                t = self.buf[k][l]
                n = t.numel() if t is not None else 1
                arr = np.frombuffer(raw[at:at + 4 * n], dtype=np.float32)
                at += 4 * n
                if t is not None:
                    t.copy_(torch.from_numpy(arr.copy()).view_as(t))
        self.refresh()


# ------------------------------------------------------------------------------------ proposal pipeline
def _bind_proposal(lib_):
    vp, i, u64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint64
    lib_.doa_synth_ula.argtypes = [i, i, i, vp, vp, i, vp, u64, u64, vp, vp]
    lib_.doa_proposal_windows.argtypes = [vp, vp, i, i, i, Grid, i, vp, vp]
    lib_.doa_scan_windows.argtypes = [vp, i, vp, vp, vp, i, i, Grid, vp, i, i, vp, vp, vp, vp, vp, vp, vp]
    lib_.doa_proposal_judge.argtypes = [vp, i, vp, vp, i, vp, Grid, Grid, vp, i, i, vp, vp, i, vp, vp, vp, vp, vp]
    for n in ("doa_synth_ula", "doa_proposal_windows", "doa_scan_windows", "doa_proposal_judge"):
        getattr(lib_, n).restype = i


def doa_synth_ula(d: torch.Tensor, angles: torch.Tensor, snr_db: torch.Tensor, M: int, N: int, seed: int,
                  first_instance: int, X: torch.Tensor, stream=None) -> None:
    """X[b] = A S + W for every row b (see include/doa.h). d int32 (B), angles float32 (B, dmax)."""
    _bind_proposal(lib())
    B, dmax = angles.shape
    _check(lib().doa_synth_ula(B, M, N, _dev(d), _dev(angles), dmax, _dev(snr_db), seed, first_instance, _dev(X),
                               _stream(stream)), "doa_synth_ula")


def doa_proposal_windows(probs: torch.Tensor, d: torch.Tensor, fine: Grid, width: int, win_first: torch.Tensor,
                         extra: int = 0, stream=None) -> None:
    _bind_proposal(lib())
    B, dmax = win_first.shape
    _check(lib().doa_proposal_windows(_dev(probs), _dev(d), B, dmax, extra, fine, width, _dev(win_first),
                                      _stream(stream)), "doa_proposal_windows")


def doa_scan_windows(B: torch.Tensor, M: int, K: torch.Tensor, d: torch.Tensor, fine: Grid, S: torch.Tensor,
                     Pwin: torch.Tensor, idx: torch.Tensor, val: torch.Tensor, count: torch.Tensor,
                     win_first: Optional[torch.Tensor] = None, width: int = 0, full: bool = False,
                     rows: Optional[torch.Tensor] = None, nrows: Optional[int] = None,
                     fallback: Optional[torch.Tensor] = None, stream=None) -> None:
    _bind_proposal(lib())
    dmax = idx.shape[1]
    n = nrows if nrows is not None else (rows.numel() if rows is not None else idx.shape[0])
    _check(lib().doa_scan_windows(_dev(B), M, _dev(K), _dev(d), _dev(rows), n, dmax, fine, _dev(win_first), width,
                                  1 if full else 0, _dev(S), _dev(Pwin), _dev(idx), _dev(val), _dev(count),
                                  _dev(fallback), _stream(stream)), "doa_scan_windows")


JUDGE_MAX = 16


def doa_proposal_judge(B: torch.Tensor, M: int, K: torch.Tensor, d: torch.Tensor, Pc: torch.Tensor, coarse: Grid,
                       fine: Grid, win_first: torch.Tensor, width: int, val: torch.Tensor, count: torch.Tensor,
                       jwidth: int, judge_first: torch.Tensor, S: torch.Tensor, Pjudge: torch.Tensor,
                       fallback: torch.Tensor, stream=None) -> None:
    """Marks in `fallback` the rows whose windowed peaks may differ from the full-grid method's
    (see include/doa.h). Pc: (batch, coarse.L) coarse spectra; judge_first: (batch, 16) int32;
    Pjudge: (batch, 16, jwidth) float32 scratch."""
    _bind_proposal(lib())
    batch, dmax = win_first.shape
    _check(lib().doa_proposal_judge(_dev(B), M, _dev(K), _dev(d), batch, _dev(Pc), coarse, fine, _dev(win_first), dmax,
                                    width, _dev(val), _dev(count), jwidth, _dev(judge_first), _dev(S), _dev(Pjudge),
                                    _dev(fallback), _stream(stream)), "doa_proposal_judge")


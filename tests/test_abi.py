"""The C ABI library builds, loads and exports every symbol include/doa.h declares; host-side
planning and argument checks behave as documented. No GPU needed (no kernel is launched)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libdoa():
    from paper_2007_14135_gb300 import build
    build.build()
    from paper_2007_14135_gb300 import doa
    return doa


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "doa.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(doa_\w+)\s*\(", src)
    return sorted(set(names))


def test_exports_every_declared_symbol(libdoa):
    declared = _declared_functions()
    assert len(declared) >= 8
    lib = ctypes.CDLL(libdoa.LIB_PATH)
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(libdoa.EXPORTS) == declared


def test_status_strings(libdoa):
    for s in range(8):
        assert libdoa.status_str(s)
    assert libdoa.status_str(99) == "unknown status"


def test_argument_errors_return_einval(libdoa):
    L = libdoa.lib()
    fake = ctypes.c_void_p(0x10000)  # never dereferenced: every call below fails its checks first
    g = libdoa.grid(-90.0, 0.1, 1801)
    assert L.doa_covariance(None, 8, 100, 100, fake, fake, 0, None) == libdoa.EINVAL
    assert L.doa_covariance(fake, 1, 100, 100, fake, fake, 0, None) == libdoa.EINVAL
    assert L.doa_covariance(fake, 65, 100, 100, fake, fake, 0, None) == libdoa.EINVAL
    assert L.doa_covariance(fake, 8, 100, 99, fake, fake, 0, None) == libdoa.EINVAL
    assert L.doa_covariance(fake, 8, 100, 100, None, None, 0, None) == libdoa.EINVAL
    assert L.doa_covariance(ctypes.c_void_p(0x10004), 8, 100, 100, fake, fake, 0, None) == libdoa.EINVAL
    assert L.doa_noise_subspace(fake, 8, 8, 1, None, fake, None, fake, None) == libdoa.EINVAL
    assert L.doa_noise_subspace(fake, 8, 2, 4, None, fake, None, fake, None) == libdoa.EINVAL
    assert L.doa_noise_subspace(fake, 8, 2, 1, None, fake, None, None, None) == libdoa.EINVAL
    assert L.doa_scan(fake, 8, 0, g, 0, fake, None) == libdoa.EINVAL
    assert L.doa_scan(fake, 8, 9, g, 0, fake, None) == libdoa.EINVAL
    assert L.doa_scan(fake, 8, 6, libdoa.grid(-90.0, 0.1, 2), 0, fake, None) == libdoa.EINVAL
    assert L.doa_scan(fake, 8, 6, libdoa.grid(-90.0, 0.0, 100), 0, fake, None) == libdoa.EINVAL
    assert L.doa_scan(fake, 8, 6, g, 7, fake, None) == libdoa.EINVAL
    assert L.doa_peaks(fake, 2, 1, fake, fake, fake, None) == libdoa.EINVAL
    assert L.doa_peaks(fake, 10, 1, None, fake, fake, None) == libdoa.EINVAL


def _prob(libdoa, M=16, N=4096, d=4, mask=0xF, L=18001, step=0.01, **kw):
    p = libdoa.Problem(0x100000, 0x200000, 0x300000, 0x400000, 0x500000, 0, libdoa.grid(-90.0, step, L),
                       M, N, N, d, mask, 0)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def test_batch_plan_layout(libdoa):
    import numpy as np
    probs = [_prob(libdoa), _prob(libdoa, M=8, N=1000, d=2, mask=0b0010, L=1801, step=0.1),
             _prob(libdoa, M=33, N=3000, d=5, mask=0b1001, L=1801, step=0.1)]
    arr = (libdoa.Problem * 3)(*probs)
    n = libdoa.lib().doa_batch_plan_bytes(arr, 3)
    assert n > 0
    buf = np.zeros(n, np.uint8)
    ws = ctypes.c_size_t(0)
    bad = ctypes.c_int(7)
    assert libdoa.lib().doa_batch_plan(arr, 3, None, buf.ctypes.data, n, ctypes.byref(ws), ctypes.byref(bad)) == 0
    assert bad.value == -1
    hdr = buf[:64].view(np.int32)
    assert hdr[0] == 0x444F4131            # magic
    # nprob, njobs, ngrids, ncov, nreduce: problems with M <= 16 take the tensor-core covariance,
    # so only the M = 33 problem has CUDA-core chunk items (3) and a partial-sum reduction
    assert list(hdr[1:6]) == [3, 4 + 1 + 2, 2, 3, 1]
    full = buf.view(np.int32)
    assert list(full[108:110]) == [1, 1]   # ncovtc: one problem with M <= 8, one with 8 < M <= 16
    off0, off1 = (int(v) for v in buf[440:456].view(np.int64))
    assert buf[off0:off0 + 4].view(np.int32)[0] == 1 and buf[off1:off1 + 4].view(np.int32)[0] == 0
    # workspace: 32- and 64-bit phase tables per grid, one int32 mark per tensor-core problem, then
    # per problem R, the covariance partials (CUDA-core problems with more than one chunk) and one
    # scan factor (M x (M+1) complex128 + M EV weights), each allocation rounded up to 256 bytes
    def factor(M):   # FP64 factor and EV weights, then the FP32 copy (padded rows), w32, thresholds
        mp = 8 if M <= 8 else 16 if M <= 16 else 32 if M <= 32 else 64
        return (M * (M + 1) * 16 + M * 8 + 15) // 16 * 16 + (M + 1) * mp * 16 + mp * 4 + 16
    need = (18001 + 1801) * 12 + 8 + (16 * 16 * 16) + factor(16) + (8 * 8 * 16) + factor(8) \
        + (33 * 33 * 16) * (1 + 3) + factor(33)
    assert ws.value >= need and ws.value < need + 256 * 12
    # too small a buffer
    assert libdoa.lib().doa_batch_plan(arr, 3, None, buf.ctypes.data, n - 1, ctypes.byref(ws), None) == libdoa.ENOMEM


def test_batch_plan_covariance_forms(libdoa):
    """The tensor-core covariance takes M <= 16 problems with a 16-byte aligned X, an even ldx and
    N <= 2^21, longest first; DOA_FLAG_COV_CUDA_CORE and the other problems keep the CUDA-core items."""
    import numpy as np
    probs = [_prob(libdoa, N=1000), _prob(libdoa, N=5000), _prob(libdoa, N=3000, flags=libdoa.FLAG_COV_CUDA_CORE),
             _prob(libdoa, M=12, N=2000, X=0x100008), _prob(libdoa, M=12, N=2000, ldx=2001),
             _prob(libdoa, M=4, N=300, d=2), _prob(libdoa, M=16, N=(1 << 21) + 2, ldx=(1 << 21) + 2)]
    arr = (libdoa.Problem * len(probs))(*probs)
    n = libdoa.lib().doa_batch_plan_bytes(arr, len(probs))
    buf = np.zeros(n, np.uint8)
    ws = ctypes.c_size_t(0)
    assert libdoa.lib().doa_batch_plan(arr, len(probs), None, buf.ctypes.data, n, ctypes.byref(ws), None) == 0
    full = buf.view(np.int32)
    assert list(full[108:110]) == [1, 2]
    off0, off1 = (int(v) for v in buf[440:456].view(np.int64))
    assert list(buf[off0:off0 + 4].view(np.int32)) == [5]
    assert list(buf[off1:off1 + 8].view(np.int32)) == [1, 0]          # N = 5000 before N = 1000
    # CUDA-core chunks: 3000 (flag), 2000 (misaligned X), 2000 (odd ldx), 2^21 + 2 (too long)
    chunks = 3 + 2 + 2 + ((1 << 21) + 2 + 1023) // 1024
    assert full[4] == chunks and full[5] == 4


@pytest.mark.parametrize("field,value", [("M", 1), ("M", 65), ("d", 16), ("d", -1), ("N", 0), ("ldx", 100),
                                         ("alg_mask", 0), ("alg_mask", 16), ("prec", 9), ("X", None)])
def test_batch_plan_rejects(libdoa, field, value):
    import numpy as np
    probs = [_prob(libdoa), _prob(libdoa, **{field: value})]
    arr = (libdoa.Problem * 2)(*probs)
    assert libdoa.lib().doa_batch_plan_bytes(arr, 2) == 0
    buf = np.zeros(1 << 16, np.uint8)
    ws = ctypes.c_size_t(0)
    bad = ctypes.c_int(-5)
    st = libdoa.lib().doa_batch_plan(arr, 2, None, buf.ctypes.data, buf.size, ctypes.byref(ws), ctypes.byref(bad))
    assert st == libdoa.EINVAL and bad.value == 1


def test_solve_batch_rejects_bad_plan(libdoa):
    import numpy as np
    junk = np.zeros(256, np.uint8)
    fake = ctypes.c_void_p(0x10000)
    assert libdoa.lib().doa_solve_batch(junk.ctypes.data, fake, fake, 1 << 20, fake, None, None) == libdoa.EINVAL


def test_batch_plan_scan_pt(libdoa):
    import numpy as np
    probs = [_prob(libdoa, M=8, N=1000, d=2, mask=0b0010, L=1801, step=0.1), _prob(libdoa, M=33, N=3000, d=5)]
    arr = (libdoa.Problem * 2)(*probs)
    n = libdoa.lib().doa_batch_plan_bytes(arr, 2)
    ws = ctypes.c_size_t(0)
    for pts, ok in [((1, 1, 1, 1), True), ((4, 4, 2, 1), True), ((2, 0, 0, 0), True), ((8, 0, 0, 0), False),
                    ((0, 0, 4, 0), False), ((0, 0, 0, 2), False)]:
        buf = np.zeros(n, np.uint8)
        tun = libdoa.Tuning((ctypes.c_int32 * 4)(*pts), (ctypes.c_int32 * 4)(0, 0, 0, 0))
        st = libdoa.lib().doa_batch_plan(arr, 2, ctypes.cast(ctypes.pointer(tun), ctypes.c_void_p), buf.ctypes.data,
                                         n, ctypes.byref(ws), None)
        assert (st == 0) == ok, pts
        if ok:
            got = buf[:128].view(np.int32)[22:26]
            want = [p if p else d for p, d in zip(pts, (4, 4, 1, 1))]
            assert list(got) == want
            tiles = buf[:128].view(np.int64)[7:11]      # scan_tiles per bucket
            # one scan job per problem: its four algorithms share the tiles of one grid pass
            assert tiles[0] == -(-1801 // (128 * want[0])) and tiles[3] == -(-18001 // 128)


def test_batch_plan_eig_mats(libdoa):
    """Matrices per Jacobi warp: allowed powers of two up to the bucket's lane budget, default by
    problem count; written to the plan header."""
    import numpy as np
    probs = [_prob(libdoa, M=8, N=1000, d=2, mask=0b0010, L=1801, step=0.1), _prob(libdoa, M=16, N=3000, d=5),
             _prob(libdoa, M=20, N=300, d=2, mask=1, L=1801, step=0.1)]
    arr = (libdoa.Problem * 3)(*probs)
    n = libdoa.lib().doa_batch_plan_bytes(arr, 3)
    ws = ctypes.c_size_t(0)
    for em, ok in [((0, 0, 0, 0), True), ((8, 4, 2, 1), True), ((1, 2, 1, 0), True), ((16, 0, 0, 0), False),
                   ((0, 8, 0, 0), False), ((0, 0, 4, 0), False), ((0, 0, 0, 2), False), ((3, 0, 0, 0), False)]:
        buf = np.zeros(n, np.uint8)
        tun = libdoa.Tuning((ctypes.c_int32 * 4)(0, 0, 0, 0), (ctypes.c_int32 * 4)(*em))
        st = libdoa.lib().doa_batch_plan(arr, 3, ctypes.cast(ctypes.pointer(tun), ctypes.c_void_p), buf.ctypes.data,
                                         n, ctypes.byref(ws), None)
        assert (st == 0) == ok, em
        if ok:
            got = list(buf[:256].view(np.int32)[58:62])
            # default with one problem per bucket: no packing
            assert got == [v if v else 1 for v in em], (em, got)


def test_batch_plan_tensor_scan_problems(libdoa):
    """Split-precision scan forms are planned into their own tensor-core list (M <= 32 only)."""
    import numpy as np
    ok = [_prob(libdoa, M=16, prec=3), _prob(libdoa, M=32, d=5, prec=2), _prob(libdoa, M=8, d=2)]
    arr = (libdoa.Problem * 3)(*ok)
    n = libdoa.lib().doa_batch_plan_bytes(arr, 3)
    assert n > 0
    buf = np.zeros(n, np.uint8)
    ws = ctypes.c_size_t(0)
    assert libdoa.lib().doa_batch_plan(arr, 3, None, buf.ctypes.data, n, ctypes.byref(ws), None) == 0
    h32 = buf[:512].view(np.int32)
    assert h32[67] == 2                       # tc_jobs
    assert h32[68] == 256                     # TMEM columns: 2 buffers x 2 accumulators x N (N = 64 for Kf = 28)
    assert list(h32[10:14]) == [1, 0, 0, 0]   # FP32 scan lists hold only the M = 8 problem
    for bad in (_prob(libdoa, M=33, prec=3), _prob(libdoa, M=16, prec=1), _prob(libdoa, M=16, prec=4)):
        arr = (libdoa.Problem * 1)(bad)
        assert libdoa.lib().doa_batch_plan_bytes(arr, 1) == 0


def test_geometry_argument_errors(libdoa):
    L = libdoa.lib()
    fake = ctypes.c_void_p(0x10000)
    az = libdoa.grid(0.0, 1.0, 360)

    def geo(pos=0x20000, Le=90, wrap=1, el_lo=1.0, el_step=1.0):
        return libdoa.Geometry(pos, el_lo, el_step, Le, wrap)

    assert L.doa_scan_geometry(fake, 8, 0, az, geo(), fake, fake, 1 << 20, None) == libdoa.EINVAL   # K < 1
    assert L.doa_scan_geometry(fake, 8, 9, az, geo(), fake, fake, 1 << 20, None) == libdoa.EINVAL        # K > M
    assert L.doa_scan_geometry(fake, 8, 6, az, geo(pos=None), fake, fake, 1 << 20, None) == libdoa.EINVAL
    assert L.doa_scan_geometry(fake, 8, 6, az, geo(pos=0x20004), fake, fake, 1 << 20, None) == libdoa.EINVAL   # 8-byte alignment
    assert L.doa_scan_geometry(fake, 8, 6, az, geo(Le=0), fake, fake, 1 << 20, None) == libdoa.EINVAL
    assert L.doa_scan_geometry(fake, 8, 6, az, geo(wrap=2), fake, fake, 1 << 20, None) == libdoa.EINVAL
    assert L.doa_scan_geometry(fake, 8, 6, az, geo(el_step=float("nan")), fake, fake, 1 << 20, None) == libdoa.EINVAL
    assert L.doa_scan_geometry(fake, 8, 6, libdoa.grid(0.0, 1.0, 0), geo(), fake, fake, 1 << 20, None) == libdoa.EINVAL
    assert L.doa_scan_geometry(fake, 8, 6, libdoa.grid(0.0, 1.0, 1 << 16), geo(Le=1 << 15), fake, fake, 1 << 20, None) == libdoa.EINVAL
    assert L.doa_scan_geometry(fake, 8, 6, az, geo(), ctypes.c_void_p(0x10002), fake, 1 << 20, None) == libdoa.EINVAL
    assert L.doa_scan_geometry(fake, 8, 6, az, geo(), fake, None, 1 << 20, None) == libdoa.EINVAL    # no scratch
    assert L.doa_scan_geometry(fake, 8, 6, az, geo(), fake, ctypes.c_void_p(0x10008), 1 << 20, None) == libdoa.EINVAL
    assert L.doa_scan_geometry(fake, 8, 6, az, geo(), fake, fake, 24 * 450 - 1, None) == libdoa.ENOMEM
    assert L.doa_scan_geometry_ws_bytes(360, 90) == 24 * 450 and L.doa_scan_geometry_ws_bytes(0, 90) == 0
    assert L.doa_peaks2d(fake, 0, 5, 0, 1, fake, fake, fake, None) == libdoa.EINVAL
    assert L.doa_peaks2d(fake, 5, 5, 3, 1, fake, fake, fake, None) == libdoa.EINVAL
    assert L.doa_peaks2d(fake, 5, 5, 0, 64, fake, fake, fake, None) == libdoa.EINVAL
    assert L.doa_peaks2d(fake, 5, 5, 0, 1, None, fake, fake, None) == libdoa.EINVAL
    assert L.doa_peaks2d(fake, 5, 5, 0, 1, fake, fake, None, None) == libdoa.EINVAL


def test_batch_plan_geometry_problems(libdoa):
    """Problems with a geometry go to their own per-bucket scan lists (tiles over La x Le points),
    need no ULA phase table, and must be FP32 without peak polish."""
    import numpy as np

    def gprob(M=8, La=360, Le=90, **kw):
        p = _prob(libdoa, M=M, N=1024, d=2, mask=0xF, L=La, step=1.0)
        p.grid = libdoa.grid(0.0, 1.0, La)
        p.geom = libdoa.Geometry(0x20000, 1.0, 1.0, Le, 1)
        for k, v in kw.items():
            setattr(p, k, v)
        return p

    probs = [gprob(), _prob(libdoa, M=8, d=2, L=1801, step=0.1), gprob(M=16, La=97, Le=13), gprob(La=1, Le=1)]
    arr = (libdoa.Problem * 4)(*probs)
    n = libdoa.lib().doa_batch_plan_bytes(arr, 4)
    assert n > 0
    buf = np.zeros(n, np.uint8)
    ws = ctypes.c_size_t(0)
    assert libdoa.lib().doa_batch_plan(arr, 4, None, buf.ctypes.data, n, ctypes.byref(ws), None) == 0
    h32 = buf[:512].view(np.int32)
    h64 = buf[:512].view(np.int64)
    assert h32[3] == 1                                  # ngrids: only the ULA problem's grid
    assert h32[96] == 3                                 # geometry grids: 360 x 90, 97 x 13, 1 x 1
    assert list(h32[10:14]) == [1, 0, 0, 0]             # ULA scan lists
    assert list(h32[76:80]) == [2, 1, 0, 0]             # geometry scan lists per M bucket
    pt = list(h32[22:26])
    assert list(h64[40:44]) == [-(-(360 * 90) // (128 * pt[0])) + 1, -(-(97 * 13) // (128 * pt[1])), 0, 0]
    assert libdoa.BatchPlan.header_index("geo_jobs") == 76
    for bad in (gprob(prec=3), gprob(flags=1), gprob(Le=0), gprob(La=0), gprob(La=1 << 16, Le=1 << 15)):
        one = (libdoa.Problem * 1)(bad)
        assert libdoa.lib().doa_batch_plan_bytes(one, 1) == 0


def test_batch_plan_optional_outputs(libdoa):
    """Refined angles, root angles and model-order outputs: counted in the plan header, the root
    form only on ULA problems, misaligned outputs rejected; the launch count follows."""
    import numpy as np

    def plan_of(probs):
        arr = (libdoa.Problem * len(probs))(*probs)
        n = libdoa.lib().doa_batch_plan_bytes(arr, len(probs))
        if n == 0:
            return None
        buf = np.zeros(n, np.uint8)
        ws = ctypes.c_size_t(0)
        assert libdoa.lib().doa_batch_plan(arr, len(probs), None, buf.ctypes.data, n, ctypes.byref(ws), None) == 0
        return buf, ws.value

    base = _prob(libdoa, M=8, d=2, L=1801, step=0.1)
    with_all = _prob(libdoa, M=8, d=2, L=1801, step=0.1, peak_angle=0x700000, root_angle=0x710000, order_est=0x720000)
    buf0, ws0 = plan_of([base])
    buf1, ws1 = plan_of([with_all, base])
    h1 = buf1[:512].view(np.int32)
    assert h1[100] == 1 and h1[101] == 1                 # nrefine, nroots
    assert buf0[:512].view(np.int32)[100] == 0
    geo = _prob(libdoa, M=8, d=2, L=360, step=1.0)
    geo.geom = libdoa.Geometry(0x20000, 1.0, 1.0, 90, 1)
    geo_ok = _prob(libdoa, M=8, d=2, L=360, step=1.0, peak_angle=0x700000, order_est=0x720000)
    geo_ok.geom = libdoa.Geometry(0x20000, 1.0, 1.0, 90, 1)
    assert plan_of([geo_ok]) is not None                 # refinement and model order on a geometry problem
    geo.root_angle = 0x710000
    assert plan_of([geo]) is None                        # the root form needs the ULA
    for field, value in (("peak_angle", 0x700004), ("root_angle", 0x710004), ("order_est", 0x720002)):
        bad = _prob(libdoa, M=8, d=2, L=1801, step=0.1, **{field: value})
        assert plan_of([bad]) is None, field
    # polish: the plan reserves one float per job for the value below the selection
    pol = _prob(libdoa, M=8, d=2, L=1801, step=0.1, flags=1)
    bufp, wsp = plan_of([pol])
    assert wsp >= ws0 + 4 * 4 - 256 and bufp[:512].view(np.int64)[51] >= 0     # next_val_off
    assert buf0[:512].view(np.int64)[51] == -1


def test_batch_plan_shared_steering_tables(libdoa):
    """Geometry problems that pass the same positions pointer with the same grid and M share one FP32
    steering table (float2[MP][ldt], ldt = La x Le rounded up to 1024) in the workspace; a problem
    alone with its key gets none."""
    import numpy as np

    def gprob(M=8, La=360, Le=90, pos=0x20000):
        p = _prob(libdoa, M=M, N=1024, d=2, mask=0xF, L=La, step=1.0)
        p.grid = libdoa.grid(0.0, 1.0, La)
        p.geom = libdoa.Geometry(pos, 1.0, 1.0, Le, 1)
        return p

    def plan_of(probs):
        arr = (libdoa.Problem * len(probs))(*probs)
        n = libdoa.lib().doa_batch_plan_bytes(arr, len(probs))
        buf = np.zeros(n, np.uint8)
        ws = ctypes.c_size_t(0)
        assert libdoa.lib().doa_batch_plan(arr, len(probs), None, buf.ctypes.data, n, ctypes.byref(ws), None) == 0
        return buf, ws.value

    shared = [gprob(), gprob(), gprob(M=16), gprob(pos=0x30000), gprob(La=97, Le=13), gprob(La=97, Le=13)]
    alone = [gprob(pos=0x20000 + 0x1000 * i) for i in range(4)] + [gprob(La=97, Le=13, pos=0x40000),
                                                                    gprob(La=97, Le=13, pos=0x41000)]
    alone[2] = gprob(M=16, pos=0x22000)
    bs, wss = plan_of(shared)
    ba, wsa = plan_of(alone)
    hs, ha = bs[:512].view(np.int32), ba[:512].view(np.int32)
    assert libdoa.BatchPlan.header_index("ngeo_steer") == 104
    assert hs[104] == 2 and ha[104] == 0                  # (pos, 360 x 90, M=8) and (pos, 97 x 13, M=8)
    assert hs[105] == 32768                                # largest row stride: 32 400 rounded up to 1024
    assert wss - wsa == 8 * 8 * 32768 + 8 * 8 * 2048        # both tables, MP = 8 rows each
    off = int(bs[:512].view(np.int64)[53])                 # off_geo_steer
    ent = bs[off:off + 80]
    assert int(ent[:8].view(np.int64)[0]) == 0x20000       # positions pointer
    geo_grid, M, MP, npts, ldt = ent[8:28].view(np.int32)
    assert (M, MP, npts, ldt) == (8, 8, 32400, 32768)
    geo_grid2, M2, MP2, npts2, ldt2 = ent[48:68].view(np.int32)
    assert (M2, MP2, npts2, ldt2) == (8, 8, 97 * 13, 2048) and geo_grid2 != geo_grid
    tab0, tab1 = int(ent[32:40].view(np.int64)[0]), int(ent[72:80].view(np.int64)[0])
    assert tab0 % 256 == 0 and tab1 >= tab0 + 8 * 8 * 32768


def test_batch_plan_many_distinct_arrays(libdoa):
    """40 000 geometry problems, each with its own positions pointer except two pairs: the plan
    finds the two shared tables among all the keys, and planning stays fast (the key lookup is a
    hash map, not a scan over the keys seen so far)."""
    import time
    import numpy as np

    n = 40000
    base = _prob(libdoa, M=8, N=256, d=2, mask=1 << 1, L=36, step=10.0)
    base.grid = libdoa.grid(0.0, 10.0, 36)
    arr = (libdoa.Problem * n)()
    for i in range(n):
        arr[i] = base
        arr[i].geom = libdoa.Geometry(0x10000000 + 64 * i, 1.0, 10.0, 9, 1)
    arr[7].geom = libdoa.Geometry(0x10000000 + 64 * 3, 1.0, 10.0, 9, 1)          # shares with problem 3
    arr[n - 1].geom = libdoa.Geometry(0x10000000 + 64 * 100, 1.0, 10.0, 9, 1)    # shares with problem 100
    t0 = time.perf_counter()
    nb = libdoa.lib().doa_batch_plan_bytes(arr, n)
    buf = np.zeros(nb, np.uint8)
    ws = ctypes.c_size_t(0)
    assert libdoa.lib().doa_batch_plan(arr, n, None, buf.ctypes.data, nb, ctypes.byref(ws), None) == 0
    elapsed = time.perf_counter() - t0
    h = buf[:512].view(np.int32)
    assert h[104] == 2 and h[105] == 1024                 # two tables, 36 x 9 points rounded up to 1024
    assert elapsed < 1.0, elapsed                          # ~15 ms measured; a key scan takes seconds


def test_binding_has_no_host_fallback(libdoa):
    """Host tensors are refused before any call reaches the library: the stages run only in the CUDA
    kernels, and there is no CPU path to fall back to."""
    import torch
    X = torch.zeros(4, 16, dtype=torch.complex64)
    R = torch.zeros(4, 4, dtype=torch.complex128)
    P = torch.zeros(181, dtype=torch.float32)
    idx = torch.zeros(2, dtype=torch.int32)
    val = torch.zeros(2, dtype=torch.float32)
    cnt = torch.zeros(1, dtype=torch.int32)
    with pytest.raises(ValueError):
        libdoa.doa_covariance(X, R64=R)
    with pytest.raises(ValueError):
        libdoa.doa_peaks(P, 2, idx, val, cnt)


def test_svd_data_argument_checks(libdoa):
    """doa_svd_data: size, pointer, alignment and parameter checks run before anything is enqueued;
    the workspace covers the FP64 rows (16 M N bytes) and grows with N."""
    L = libdoa.lib()
    fake = ctypes.c_void_p(0x10000)
    big = 1 << 40
    assert L.doa_svd_data_ws_bytes(1, 100) == 0 and L.doa_svd_data_ws_bytes(65, 100) == 0
    assert L.doa_svd_data_ws_bytes(16, 0) == 0
    n1, n2 = L.doa_svd_data_ws_bytes(16, 1000), L.doa_svd_data_ws_bytes(16, 2000)
    assert n1 >= 16 * 16 * 1000 and n2 - n1 == 16 * 16 * 1000
    ok = (fake, 0, 16, 1000, 1000, 1e-15, 60, fake, fake, fake, fake, big, None)
    for k, bad in ((0, None), (2, 1), (2, 65), (3, 0), (4, 999), (5, 0.0), (5, float("nan")), (6, 0), (6, 1001),
                   (7, None), (8, None), (9, None), (10, None), (1, 2),
                   (0, ctypes.c_void_p(0x10004)),              # complex64 X: 8-byte aligned
                   (8, ctypes.c_void_p(0x10008))):             # U: 16-byte aligned
        args = list(ok)
        args[k] = bad
        assert L.doa_svd_data(*args) == libdoa.EINVAL, (k, bad)
    args = list(ok)
    args[1], args[0] = 1, ctypes.c_void_p(0x10008)             # complex128 X: 16-byte aligned
    assert L.doa_svd_data(*args) == libdoa.EINVAL
    args = list(ok)
    args[11] = n1 - 1
    assert L.doa_svd_data(*args) == libdoa.ENOMEM

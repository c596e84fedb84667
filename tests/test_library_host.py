"""Host-side checks of the C-ABI library (no GPU needed): it builds, loads, exports every
entry point its header declares, and its host-only logic is right."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1403_3746_gb300 as lbm
from paper_1403_3746_gb300 import build as lbm_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    lbm_build.build()
    return lbm.lib()


def declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 18
    for n in names:
        assert hasattr(L, n), n


def test_default_params_are_the_phase_separation_set(L):
    p = lbm.default_params()
    assert (p.tau, p.dt, p.dx, p.dy, p.K, p.H, p.q, p.zeta, p.b, p.eta0) == \
        (1e-4, 1e-4, 1 / 256, 1 / 256, 5e-6, 0.0, -0.004, 0.0, 2.0, 2.5)
    assert p.precision == lbm.LBM_FP64 and p.flags == 0


def test_maxwell_matches_oracle_construction(L):
    # the library solves equal pressure + equal chemical potential; the oracle the equal-area rule
    from oracle.maxwell import coexistence
    for T in (0.8, 0.85, 0.9, 0.95, 0.99):
        rl, rv = lbm.maxwell(T)
        ol, ov = coexistence(T)
        assert rl == pytest.approx(ol, rel=1e-11) and rv == pytest.approx(ov, rel=1e-10)
    with pytest.raises(lbm.LbmError):
        lbm.maxwell(1.2)


@pytest.mark.parametrize("nx,ny", [(3, 8), (8, 0), (8, 6), (8192, 8), (1, 8)])
def test_create_rejects_bad_sizes_before_touching_the_device(L, nx, ny):
    p = lbm.default_params()
    h = ctypes.c_void_p()
    assert L.lbm_create(nx, ny, ctypes.byref(p), None, ctypes.byref(h)) == -1
    assert not h.value


@pytest.mark.parametrize("field,value", [("tau", 0.0), ("dt", -1.0), ("dx", float("nan")),
                                         ("precision", 7), ("flags", 64)])
def test_create_rejects_bad_params(L, field, value):
    p = lbm.default_params(**{field: value})
    h = ctypes.c_void_p()
    assert L.lbm_create(16, 16, ctypes.byref(p), None, ctypes.byref(h)) == -1


def test_error_strings(L):
    assert L.lbm_strerror(0) == b"ok"
    assert L.lbm_strerror(-7).startswith(b"unsupported")
    assert L.lbm_strerror(-99) == b"unknown error"


@pytest.mark.parametrize("sizes", [[], [(16, 16), (24, 16)], [(16, 16), (16, 8192)], [(2, 1)]])
def test_batch_create_rejects_bad_sizes_before_touching_the_device(L, sizes):
    p = lbm.default_params()
    n = max(len(sizes), 1)
    nx = (ctypes.c_int * n)(*[s[0] for s in sizes])
    ny = (ctypes.c_int * n)(*[s[1] for s in sizes])
    h = ctypes.c_void_p()
    assert L.lbm_batch_create(len(sizes), nx, ny, ctypes.byref(p), None, ctypes.byref(h)) == -1
    assert not h.value
    assert L.lbm_batch_count(None) == 0


@pytest.mark.parametrize("kw", [dict(keff_terms=0), dict(keff_terms=9), dict(flags=16),
                                dict(flags=16, T_iso=-1.0), dict(flags=16, T_iso=float("inf")),
                                dict(flags=32)])
def test_create_rejects_bad_variant_params(L, kw):
    p = lbm.default_params(**kw)
    h = ctypes.c_void_p()
    assert L.lbm_create(16, 16, ctypes.byref(p), None, ctypes.byref(h)) == -1
    assert not h.value


def test_variant_defaults(L):
    p = lbm.default_params()
    assert p.keff_terms == 8 and p.T_iso == 0.0 and p.reserved == 0
    assert p.filter_alpha == 0.0 and p.filter_p == 36.0
    assert ctypes.sizeof(lbm.lbm_params) == 12 * 8 + 2 * 4 + 8 + 2 * 4 + 2 * 8


@pytest.mark.parametrize("kw", [dict(filter_alpha=-1.0), dict(filter_p=0.0), dict(filter_alpha=float("nan"))])
def test_create_rejects_bad_filter_params(L, kw):
    p = lbm.default_params(**kw)
    h = ctypes.c_void_p()
    assert L.lbm_create(16, 16, ctypes.byref(p), None, ctypes.byref(h)) == -1
    assert not h.value


def test_moments_out_arrays_are_checked():
    from paper_1403_3746_gb300 import _host_out
    assert [a.shape for a in _host_out(None, (4, 8))] == [(4, 8)] * 4
    good = [np.zeros((4, 8)) for _ in range(4)]
    assert _host_out(good, (4, 8)) == good
    ro = np.zeros((4, 8))
    ro.flags.writeable = False
    for bad in (good[:3], [np.zeros((4, 8), np.float32)] + good[1:], [np.zeros((8, 4))] + good[1:],
                [ro] + good[1:], [np.zeros((4, 16))[:, ::2]] + good[1:]):
        with pytest.raises(ValueError, match="four writable"):
            _host_out(bad, (4, 8))


def test_surface_tension_and_equimolar_radius_reducers():
    # host-side reducers of the Laplace check, against closed forms
    from paper_1403_3746_gb300.accuracy import equimolar_radius, surface_tension
    n, dx, K, w, a = 256, 1 / 256, 5e-6, 3.0, 0.6
    x = np.arange(n)
    prof = 1.0 + a * (np.tanh((x - 64) / w) - np.tanh((x - 192) / w))
    # integral of (a/w)^2 sech^4(x/w) over x (cells) is (a/w)^2 w 4/3; per unit length: / dx
    assert surface_tension(prof, dx, K) == pytest.approx(K * (a / w) ** 2 * w * 4 / 3 / dx, rel=1e-8)
    Y, X = np.mgrid[0:128, 0:128]
    rho = 0.4 + 1.2 * (np.hypot(X - 63.5, Y - 63.5) < 20.0)
    assert equimolar_radius(rho, 1.6, 0.4) == pytest.approx(20.0, rel=2e-2)
    assert equimolar_radius(np.full((8, 8), 0.4), 1.6, 0.4) == 0.0


def _line_G(n):
    # threads per line of the register FFT engine: 16 points per thread (all points for n < 16)
    return n // 16 if n >= 16 else 1


@pytest.mark.parametrize("precision", [lbm.LBM_FP64, lbm.LBM_MIXED, lbm.LBM_MIXED_RHO64])
def test_launch_plan_of_every_size_fits_the_kernels(L, precision):
    # host-side launch plan (no device) of every supported grid: each pass's CTA within its
    # thread and shared-memory limits, tiles and row groups dividing the grid, and the
    # separate-row-pass / serial-macro forms only where the kernels implement them (float64
    # rows of 4096)
    es = 8 if precision == lbm.LBM_FP64 else 4
    sizes = [1 << k for k in range(1, 13)]
    for nx in sizes:
        for ny in sizes:
            pl = lbm.launch_plan(nx, ny, precision)
            cap_smem = pl["cta_smem_cap"]
            assert cap_smem == 232448
            assert nx % pl["col_width"] == 0 and pl["col_width"] >= 2
            assert pl["col_threads"] == (pl["col_width"] // 2) * _line_G(ny) <= pl["pass_thread_cap"]
            for k in ("col_smem", "macro_smem", "update_smem", "rowd_smem"):
                assert 0 <= pl[k] <= cap_smem, (nx, ny, k, pl)
            for k in ("macro_rows", "update_rows", "rowd_rows"):
                assert ny % pl[k] == 0, (nx, ny, k)
            assert pl["macro_threads"] <= pl["macro_thread_cap"]
            assert pl["rowd_threads"] <= (384 if es == 8 else 768)
            special = es == 8 and nx == 4096
            assert pl["update_ax"] == (1 if special else 0), (nx, ny, pl)
            assert pl["macro_serial"] == (1 if special else 0), (nx, ny, pl)
            # a cluster of four CTAs splits float32 rows of 4096 in the update pass
            assert pl["update_ctas_per_row"] == (4 if (es == 4 and nx == 4096) else 1), (nx, ny, pl)
            assert pl["col_ctas_per_cluster"] == 1
            if not pl["update_ax"]:
                # six line buffers per row of the update CTA, each its share of the row
                part = nx // pl["update_ctas_per_row"]
                line = (part + part // 16 + 2) * 2 * es
                assert pl["update_smem"] == 6 * pl["update_rows"] * line


@pytest.mark.parametrize("precision", [lbm.LBM_MIXED, lbm.LBM_FP64])
def test_column_tile_line_buffers_take_disjoint_banks(L, precision):
    # a column tile's L = W/2 lines share warps (line index fastest); an 8-byte (16-byte) shared
    # access is served per half-warp (quarter-warp), where each line covers 128/L bytes, so
    # consecutive line buffers must start 128/L bytes apart modulo 128 (one element at least)
    # and hold the padded line (N + N/16 complex values)
    es = 8 if precision == lbm.LBM_FP64 else 4
    cs = 2 * es
    for ly in range(1, 13):
        ny = 1 << ly
        nx = 4096 if precision == lbm.LBM_MIXED else 1024
        pl = lbm.launch_plan(nx, ny, precision)
        W, clu = pl["col_width"], pl["col_ctas_per_cluster"]
        lines = W // 2
        if lines < 2:
            continue
        stride = pl["col_smem"] // lines  # bytes per line buffer
        assert pl["col_smem"] % lines == 0
        part = ny // clu
        assert stride >= (part + part // 16) * cs, (ny, pl)
        assert stride % 128 == max(128 // lines, cs) % 128, (ny, W, stride)
        # the lines of one half-warp (quarter-warp) start at distinct offsets modulo 128 bytes
        per = 16 if es == 4 else 8  # lanes served together
        group = min(lines, per)
        assert len({(l * stride) % 128 for l in range(group)}) == group, (ny, W, stride)


def test_launch_plan_rejects_bad_sizes(L):
    for nx, ny in ((3, 8), (8, 8192), (1, 2)):
        with pytest.raises(lbm.LbmError, match="power of two"):
            lbm.launch_plan(nx, ny)
    with pytest.raises(lbm.LbmError, match="precision"):
        lbm.launch_plan(8, 8, 7)


def test_state_blob_size_and_params_hash(L):
    # header of 64 bytes, then per row 16 distributions + 4 moments in the storage precision
    assert lbm.state_bytes(64, 32, lbm.LBM_FP64) == 64 + 32 * 20 * 64 * 8
    assert lbm.state_bytes(64, 32, lbm.LBM_MIXED) == 64 + 32 * 20 * 64 * 4
    assert lbm.state_bytes(64, 32, lbm.LBM_MIXED_RHO64) == lbm.state_bytes(64, 32, lbm.LBM_MIXED)
    assert lbm.state_bytes(63, 32) == 0 and lbm.state_bytes(64, 32, 7) == 0
    a, b = lbm.default_params(), lbm.default_params()
    assert lbm.params_hash(a) == lbm.params_hash(b) != 0
    for field, value in (("tau", 2e-4), ("K", 5.000001e-6), ("precision", lbm.LBM_MIXED),
                         ("precision", lbm.LBM_MIXED_RHO64), ("flags", 8),
                         ("keff_terms", 4), ("win_alpha", 36.0), ("filter_alpha", 36.0)):
        c = lbm.default_params(**{field: value})
        assert lbm.params_hash(c) != lbm.params_hash(a), field
    # FNV-1a over the field bytes, least significant first, written out here independently
    import struct
    h = 1469598103934665603
    raw = struct.pack("<12d", a.tau, a.dt, a.dx, a.dy, a.K, a.H, a.q, a.zeta, a.b, a.eta0, a.win_alpha, a.win_p)
    raw += struct.pack("<ii", a.precision, a.flags) + struct.pack("<d", a.T_iso)
    raw += struct.pack("<ii", a.keff_terms, a.reserved) + struct.pack("<dd", a.filter_alpha, a.filter_p)
    for byte in raw:
        h = ((h ^ byte) * 1099511628211) % (1 << 64)
    assert lbm.params_hash(a) == h

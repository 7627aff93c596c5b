"""C-ABI checks that need no GPU: the library loads, exports every entry
point the header declares, validates arguments on the host, and its host
logic (grouping, scratch sizing) behaves."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2505_14372_b300 import _lib
from paper_2505_14372_b300.api import Geometry, make_groups, scratch_bytes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ptycho.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ptycho_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = C.CDLL(_lib.LIB_PATH)
    names = declared_functions()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # and the binding declares a signature for each of them
    assert not [n for n in names if n not in _lib.SIGNATURES]


def test_version_and_error_channel():
    lib = _lib.lib()
    assert b"sm_103a" in lib.ptycho_version()
    g = _lib.Geom(1, 1, 96, 96, 128, 128, 0.1, 0.0197, None, 0.66, 0, 1e-3, 0.0, 0)
    h = C.c_void_p()
    rc = lib.ptycho_create(C.byref(g), 4, 0, C.byref(h))
    assert rc == _lib.EINVAL and not h.value
    assert b"96" in lib.ptycho_last_error()


@pytest.mark.parametrize("bad", [
    dict(S=0), dict(K=0), dict(N=100), dict(H=32), dict(dx=0.0), dict(lam=-1.0),
    dict(loss="poisson", eps=0.0), dict(loss="amplitude", eps=0.0, c=0.0), dict(c=-1.0),
])
def test_geometry_validation(bad):
    args = dict(S=2, K=2, N=64, H=80, W=80, dz=(10.0,), loss="amplitude", eps=1e-3, c=0.0)
    args.update(bad)
    if args["S"] != 2:
        args["dz"] = tuple([10.0] * max(args["S"] - 1, 0))
    geom = Geometry(**args)
    g, _dz = geom.to_c()
    h = C.c_void_p()
    assert _lib.lib().ptycho_create(C.byref(g), 4, 0, C.byref(h)) == _lib.EINVAL


def test_null_dz_rejected():
    g = _lib.Geom(3, 1, 64, 64, 80, 80, 0.1, 0.0197, None, 0.66, 0, 1e-3, 0.0, 0)
    h = C.c_void_p()
    assert _lib.lib().ptycho_create(C.byref(g), 4, 0, C.byref(h)) == _lib.EINVAL


def test_null_context_calls_fail_cleanly():
    lib = _lib.lib()
    assert lib.ptycho_forward(None, None, None, None, 1, None, None) == _lib.EINVAL
    assert lib.ptycho_check(None, None) == _lib.EINVAL
    assert lib.ptycho_destroy(None) == _lib.OK


def test_scratch_bytes_store_vs_recompute():
    geom = Geometry(S=20, K=8, N=192, H=1024, W=1024, dz=tuple([10.0] * 19), loss="poisson", eps=0.8)
    store = scratch_bytes(geom, 512, "store")
    rec = scratch_bytes(geom, 512, "recompute")
    waves = 512 * 8 * 20 * 192 * 192 * 8
    assert store >= waves and rec < store - waves // 2


@pytest.mark.parametrize("mode", ["sparse", "compact"])
def test_groups_are_permutations_and_deterministic(mode):
    pos = np.stack(np.meshgrid(np.arange(20) * 3.0, np.arange(25) * 3.0, indexing="ij"), -1).reshape(-1, 2)
    P = len(pos)
    a = make_groups(P, 64, seed=7, iteration=3, mode=mode, pos=pos)
    b = make_groups(P, 64, seed=7, iteration=3, mode=mode, pos=pos)
    c = make_groups(P, 64, seed=7, iteration=4, mode=mode, pos=pos)
    assert np.array_equal(np.sort(a), np.arange(P))
    assert np.array_equal(a, b) and not np.array_equal(a, c)


def test_compact_groups_are_spatially_compact():
    pos = np.stack(np.meshgrid(np.arange(32) * 4.0, np.arange(32) * 4.0, indexing="ij"), -1).reshape(-1, 2)
    P, B = len(pos), 64
    comp = make_groups(P, B, seed=1, iteration=0, mode="compact", pos=pos)
    sparse = make_groups(P, B, seed=1, iteration=0, mode="sparse", pos=pos)

    def spread(order):
        return np.mean([np.ptp(pos[order[i:i + B]], axis=0).sum() for i in range(0, P, B)])
    assert spread(comp) < 0.5 * spread(sparse)


def test_reduced_precision_halves_store_scratch():
    # 16-bit entry-wave copies take half the bytes of complex64 ones
    geom = Geometry(S=5, K=2, N=64, H=80, W=80, dz=(10.0,) * 4)
    full = scratch_bytes(geom, 64, "store")
    geom.wave_prec = "bf16"
    half = scratch_bytes(geom, 64, "store")
    waves = 64 * 2 * 5 * 64 * 64 * 8
    assert full - half == pytest.approx(waves / 2, abs=512)


def test_static_forward_host_validation():
    """ptycho_forward_static rejects bad geometry, too many slices and
    problems larger than its fixed scratch on the host, before any device
    work (so these need no GPU)."""
    lib = _lib.lib()
    fake = C.c_void_p(16)  # never dereferenced: every case fails validation first

    def call(geom, B=4):
        g, _dz = geom.to_c()
        return lib.ptycho_forward_static(C.byref(g), fake, fake, fake, B, fake, None, None)

    assert call(Geometry(S=1, K=1, N=100, H=128, W=128)) == _lib.EINVAL
    assert call(Geometry(S=2, K=1, N=64, H=80, W=80, dz=(float("nan"),))) == _lib.EINVAL
    assert call(Geometry(S=70, K=1, N=64, H=80, W=80, dz=(10.0,) * 69)) == _lib.EINVAL
    assert b"at most 65 slices" in lib.ptycho_last_error()
    assert call(Geometry(S=1, K=8, N=256, H=300, W=300), B=64) == _lib.EINVAL
    assert b"static scratch" in lib.ptycho_last_error()
    assert call(Geometry(S=1, K=1, N=64, H=80, W=80), B=-1) == _lib.EINVAL
    assert call(Geometry(S=1, K=1, N=64, H=80, W=80), B=0) == _lib.OK


def test_deterministic_flag_validation():
    """The deterministic flag needs the recomputed-wave FFT path with FP32
    entry waves; the checks run on the host."""
    lib = _lib.lib()
    h = C.c_void_p()
    for bad in (dict(waves="store"), dict(wave_prec="bf16"), dict(dft="tf32x3", N=192, H=200, W=200)):
        args = dict(S=1, K=1, N=64, H=80, W=80, deterministic=True)
        args.update(bad)
        g, _dz = Geometry(**args).to_c()
        assert lib.ptycho_create(C.byref(g), 4, 0, C.byref(h)) == _lib.EINVAL
        assert b"deterministic" in lib.ptycho_last_error()
    g, _dz = Geometry(S=1, K=1, N=64, H=80, W=80).to_c()
    g.deterministic = 2
    assert lib.ptycho_create(C.byref(g), 4, 0, C.byref(h)) == _lib.EINVAL


def test_checked_build_exports_the_same_entry_points():
    """The checked build (index checks in the kernels, PTYCHO_ECHECK) is the
    same C-ABI: every symbol of the normal library, and ptycho_build_checked
    telling the two apart (host-only calls, no GPU needed)."""
    here = os.path.join(ROOT, "paper_2505_14372_b300")
    normal, checked = os.path.join(here, "libptycho.so"), os.path.join(here, "libptycho_checked.so")
    assert os.path.exists(checked), "build it with python -m paper_2505_14372_b300.build --checked"
    ln, lc = C.CDLL(normal), C.CDLL(checked)
    missing = [n for n in declared_functions() if not hasattr(lc, n)]
    assert not missing, missing
    ln.ptycho_build_checked.restype = C.c_int32
    lc.ptycho_build_checked.restype = C.c_int32
    assert ln.ptycho_build_checked() == 0 and lc.ptycho_build_checked() == 1

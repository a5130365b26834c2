"""Host-only checks of the C ABI (no GPU compute):

  * libac.so builds for sm_103a, loads, and exports every function that
    include/ac.h declares;
  * argument validation returns AC_ERR_ARG before any CUDA call;
  * the library's host-side forcing draw agrees with the oracle's
    independently written draw (integer wave vector bit-exact);
  * ac_strerror covers every code.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2103_01597_gb300 import build, ac
    build.build()
    return ac


def _declared():
    names = []
    for hdr in os.listdir(os.path.join(ROOT, "include")):
        if hdr.endswith(".h"):
            text = open(os.path.join(ROOT, "include", hdr)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(ac_\w+)\s*\(", text)
    return sorted(set(names))


def test_exports_every_declared_symbol(lib):
    L = ctypes.CDLL(lib.LIB_PATH)
    names = _declared()
    assert "ac_integrate_substep" in names and len(names) >= 20
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_argument_validation_without_gpu(lib):
    L = lib.load_library()
    h = ctypes.c_void_p()
    p = lib.make_params()
    for bad in [lib.make_grid((0, 4, 4)), lib.make_grid((4, 4, 4), L=(0, 1, 1)),
                lib.make_grid((4, 4, 4), layout=7)]:
        assert L.ac_init(ctypes.byref(h), ctypes.byref(bad), ctypes.byref(p), None) == lib.AC_ERR_ARG
    g = lib.make_grid((4, 4, 4))
    for bp in [lib.make_params(gamma=1.0), lib.make_params(cp=0.0), lib.make_params(nu=-1),
               lib.make_params(precision=9), lib.make_params(nu=float("nan"))]:
        assert L.ac_init(ctypes.byref(h), ctypes.byref(g), ctypes.byref(bp), None) == lib.AC_ERR_ARG
    assert L.ac_init(None, ctypes.byref(g), ctypes.byref(p), None) == lib.AC_ERR_ARG
    assert L.ac_integrate_substep(None, 1e-3, 0) == lib.AC_ERR_ARG
    assert L.ac_quit(None) == lib.AC_OK
    # the allocation-free reduction checks grid and parameters as ac_init does,
    # before any CUDA call (an infinite box length would make every derivative 0)
    fake = [8 * (q + 1) for q in range(8)]
    for bad in [lib.make_grid((4, 4, 4), L=(float("inf"), 1, 1)), lib.make_grid((0, 4, 4)),
                lib.make_grid((4, 4, 8193))]:
        with pytest.raises(lib.AcError) as ei:
            lib.ac_reduce_noalloc(fake, bad, p, lib.AC_MAX, lib.AC_UX)
        assert ei.value.code == lib.AC_ERR_ARG
    with pytest.raises(lib.AcError) as ei:
        lib.ac_reduce_noalloc(fake, g, lib.make_params(eta=float("inf")), lib.AC_MAX, lib.AC_UX)
    assert ei.value.code == lib.AC_ERR_ARG
    # the bounded-wait diagnostic checks its limit before touching the device
    assert lib.ac_diag_wait_timeout(0) == lib.AC_ERR_ARG
    assert lib.ac_diag_wait_timeout((1 << 18) + 1) == lib.AC_ERR_ARG
    # the exp diagnostic checks its arguments before touching the device
    assert L.ac_diag_exp_table(None, -1, None, None) == lib.AC_ERR_ARG
    assert L.ac_diag_exp_table(None, 5, None, None) == lib.AC_ERR_ARG
    assert L.ac_diag_exp_table(None, 0, None, None) == lib.AC_OK
    # the normal build does not check global indices and says so
    assert lib.ac_bounds_check_take() == (lib.AC_ERR_STATE, 0)
    assert lib.ac_bounds_check_selftest() == (lib.AC_ERR_STATE, [0, 0])
    assert L.ac_bounds_check_take(None) == lib.AC_ERR_ARG


def test_strerror(lib):
    for c in range(0, -7, -1):
        assert lib.ac_strerror(c).startswith("AC_")
    assert "unknown" in lib.ac_strerror(-99)


def test_forcing_draw_matches_oracle(lib, oracle_lib):
    from oracle import core
    for seed in (0, 2, 12345, 2 ** 63 + 7):
        for step in range(0, 200, 7):
            k, e, phi = lib.ac_forcing_draw(seed, step)
            fo = core.forcing_draw(seed, step, 1.0)
            assert k == fo.k
            assert max(abs(a - b) for a, b in zip(e, fo.e)) <= 1e-15
            assert abs(phi - fo.phi) <= 1e-15

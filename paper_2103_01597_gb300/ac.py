"""ctypes binding of ``libac.so`` (declared in ``include/ac.h``).

Same names as the C ABI; this module only marshals arguments.  Every step of
the substep runs in the library's CUDA kernels.  PyTorch is used for device
memory (``Simulation`` binds torch tensors with ``ac_bind_buffers``) and for
the CUDA stream.  Loading fails loudly if the compiled library is missing:
there is no CPU fallback.
"""
import ctypes
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libac.so")

AC_OK = 0
AC_ERR_ARG = -1
AC_ERR_CUDA = -2
AC_ERR_OOM = -3
AC_ERR_NONFINITE = -4
AC_ERR_TIMEOUT = -5
AC_ERR_STATE = -6

AC_LNRHO, AC_UX, AC_UY, AC_UZ, AC_SS, AC_AX, AC_AY, AC_AZ = range(8)
AC_NFIELDS = 8
AC_ALL = -1

AC_FP64, AC_FP32, AC_FP32_W64 = 0, 1, 2
AC_LAYOUT_PERIODIC, AC_LAYOUT_PADDED = 0, 1
AC_MAX, AC_MIN, AC_SUM, AC_RMS = 0, 1, 2, 3
AC_STENCIL_AUTO, AC_STENCIL_FP64, AC_STENCIL_FIXED = 0, 1, 2
AC_STENCIL_MODE_GROUP, AC_STENCIL_MODE_FIELD, AC_STENCIL_MODE_PLAIN = 0, 1, 2
AC_CONV_TCGEN05, AC_CONV_MMA_SYNC, AC_CONV_TCGEN05_PAIR = 0, 1, 2
AC_TILE_32X8, AC_TILE_16X16 = 0, 1
AC_Q_UMAG, AC_Q_EKIN, AC_Q_EMAG, AC_Q_CFL = 8, 9, 10, 11


class ac_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("lx", ctypes.c_double), ("ly", ctypes.c_double), ("lz", ctypes.c_double),
                ("layout", ctypes.c_int)]


class ac_params(ctypes.Structure):
    _fields_ = [("nu", ctypes.c_double), ("eta", ctypes.c_double), ("cs0", ctypes.c_double),
                ("gamma", ctypes.c_double), ("cp", ctypes.c_double), ("lnrho0", ctypes.c_double),
                ("force_amp", ctypes.c_double), ("seed", ctypes.c_ulonglong),
                ("precision", ctypes.c_int)]


class ac_box(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("lx", ctypes.c_double), ("ly", ctypes.c_double), ("lz", ctypes.c_double),
                ("nu", ctypes.c_double), ("eta", ctypes.c_double)]


AC_BATCH_MAX_BOXES = 128


class AcError(RuntimeError):
    def __init__(self, code, where, value=None):
        self.code = code
        self.value = value
        msg = "%s failed: %s" % (where, ac_strerror(code))
        if code == AC_ERR_CUDA or code == AC_ERR_OOM:
            msg += " (%s)" % ac_last_cuda_error()
        super().__init__(msg)


_lib = None
_c = ctypes
_vp = ctypes.c_void_p
_pd = ctypes.POINTER(ctypes.c_double)


def load_library(path=None):
    """Load libac.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise OSError("libac.so not found at %s: build it with "
                      "paper_2103_01597_gb300.build.build()" % p)
    L = ctypes.CDLL(p)
    sig = {
        "ac_init": ([ctypes.POINTER(_vp), ctypes.POINTER(ac_grid), ctypes.POINTER(ac_params), _vp],
                    _c.c_int),
        "ac_quit": ([_vp], _c.c_int),
        "ac_set_stream": ([_vp, _vp], _c.c_int),
        "ac_bind_buffers": ([_vp, ctypes.POINTER(_vp)], _c.c_int),
        "ac_field_elems": ([_vp, ctypes.POINTER(ctypes.c_size_t)], _c.c_int),
        "ac_load": ([_vp, _c.c_int, _vp], _c.c_int),
        "ac_store": ([_vp, _c.c_int, _vp], _c.c_int),
        "ac_load_w": ([_vp, _c.c_int, _vp], _c.c_int),
        "ac_store_w": ([_vp, _c.c_int, _vp], _c.c_int),
        "ac_load_f32": ([_vp, _c.c_int, _vp], _c.c_int),
        "ac_store_f32": ([_vp, _c.c_int, _vp], _c.c_int),
        "ac_integrate_substep": ([_vp, _c.c_double, _c.c_int], _c.c_int),
        "ac_integrate_step": ([_vp, _c.c_double], _c.c_int),
        "ac_periodic_halo": ([_vp], _c.c_int),
        "ac_last_cfl": ([_vp, _pd], _c.c_int),
        "ac_set_stencil_mode": ([_vp, _c.c_int], _c.c_int),
        "ac_get_stencil_path": ([_vp, ctypes.POINTER(_c.c_int)], _c.c_int),
        "ac_get_stencil_modes": ([_vp, ctypes.POINTER(_c.c_ulonglong)], _c.c_int),
        "ac_diag_fma_rate": ([_c.c_int, _pd, _vp], _c.c_int),
        "ac_set_kernel_timing": ([_vp, _c.c_int], _c.c_int),
        "ac_kernel_timings": ([_vp, _pd, _pd, ctypes.POINTER(_c.c_int)], _c.c_int),
        "ac_decomp_init": ([ctypes.POINTER(_vp), ctypes.POINTER(ac_grid),
                            ctypes.POINTER(ac_params), ctypes.POINTER(_c.c_int), _vp], _c.c_int),
        "ac_decomp_quit": ([_vp], _c.c_int),
        "ac_decomp_load": ([_vp, _c.c_int, _vp], _c.c_int),
        "ac_decomp_store": ([_vp, _c.c_int, _vp], _c.c_int),
        "ac_decomp_load_w": ([_vp, _c.c_int, _vp], _c.c_int),
        "ac_decomp_store_w": ([_vp, _c.c_int, _vp], _c.c_int),
        "ac_decomp_integrate_substep": ([_vp, _c.c_double, _c.c_int], _c.c_int),
        "ac_decomp_integrate_step": ([_vp, _c.c_double], _c.c_int),
        "ac_decomp_set_overlap": ([_vp, _c.c_int], _c.c_int),
        "ac_decomp_info": ([_vp, ctypes.POINTER(_c.c_int), ctypes.POINTER(_c.c_int),
                            ctypes.POINTER(_c.c_int), ctypes.POINTER(_c.c_ulonglong)], _c.c_int),
        "ac_decomp_partition": ([_c.c_int, ctypes.POINTER(_c.c_int)], _c.c_int),
        "ac_decomp_coord": ([ctypes.POINTER(_c.c_int), _c.c_int, ctypes.POINTER(_c.c_int)],
                            _c.c_int),
        "ac_decomp_segment": ([ctypes.POINTER(_c.c_int), _c.c_int, ctypes.POINTER(_c.c_int),
                               ctypes.POINTER(_c.c_int), ctypes.POINTER(_c.c_int),
                               ctypes.POINTER(_c.c_int)], _c.c_int),
        "ac_reduce": ([_vp, _c.c_int, _c.c_int, _pd], _c.c_int),
        "ac_forcing_draw": ([_c.c_ulonglong, _c.c_ulonglong, ctypes.POINTER(_c.c_int), _pd, _pd],
                            _c.c_int),
        "ac_set_forcing": ([_vp, ctypes.POINTER(_c.c_int), _pd, _c.c_double], _c.c_int),
        "ac_get_step": ([_vp, ctypes.POINTER(_c.c_ulonglong), ctypes.POINTER(_c.c_int)], _c.c_int),
        "ac_set_step": ([_vp, _c.c_ulonglong, _c.c_int], _c.c_int),
        "ac_launch_count": ([_vp, ctypes.POINTER(_c.c_ulonglong)], _c.c_int),
        "ac_reduce_noalloc": ([ctypes.POINTER(_vp), ctypes.POINTER(ac_grid),
                               ctypes.POINTER(ac_params), _c.c_int, _c.c_int, _pd, _vp], _c.c_int),
        "ac_batch_init": ([ctypes.POINTER(_vp), _c.c_int, ctypes.POINTER(ac_box),
                           ctypes.POINTER(ac_params), _vp], _c.c_int),
        "ac_batch_quit": ([_vp], _c.c_int),
        "ac_batch_load": ([_vp, _c.c_int, _c.c_int, _vp], _c.c_int),
        "ac_batch_store": ([_vp, _c.c_int, _c.c_int, _vp], _c.c_int),
        "ac_batch_load_w": ([_vp, _c.c_int, _c.c_int, _vp], _c.c_int),
        "ac_batch_store_w": ([_vp, _c.c_int, _c.c_int, _vp], _c.c_int),
        "ac_batch_load_f32": ([_vp, _c.c_int, _c.c_int, _vp], _c.c_int),
        "ac_batch_store_f32": ([_vp, _c.c_int, _c.c_int, _vp], _c.c_int),
        "ac_batch_integrate_substep": ([_vp, _c.c_double, _c.c_int], _c.c_int),
        "ac_batch_integrate_step": ([_vp, _c.c_double], _c.c_int),
        "ac_batch_set_graph": ([_vp, _c.c_int], _c.c_int),
        "ac_batch_tune": ([_vp, _c.c_double, _c.c_char_p, ctypes.POINTER(_c.c_int)], _c.c_int),
        "ac_batch_set_tiling": ([_vp, _c.c_int, ctypes.POINTER(_c.c_int)], _c.c_int),
        "ac_batch_get_tiling": ([_vp, ctypes.POINTER(_c.c_int), ctypes.POINTER(_c.c_int),
                                 ctypes.POINTER(_c.c_float)], _c.c_int),
        "ac_batch_reduce": ([_vp, _c.c_int, _c.c_int, _c.c_int, _pd], _c.c_int),
        "ac_batch_info": ([_vp, ctypes.POINTER(_c.c_longlong), ctypes.POINTER(_c.c_int),
                           ctypes.POINTER(_c.c_int), ctypes.POINTER(_c.c_int),
                           ctypes.POINTER(_c.c_ulonglong)], _c.c_int),
        "ac_set_stencil_order": ([_vp, _c.c_int], _c.c_int),
        "ac_set_entropy_terms": ([_vp, _c.c_double, _c.c_double, _c.c_double, _c.c_double],
                                 _c.c_int),
        "ac_get_stencil_order": ([_vp, ctypes.POINTER(_c.c_int)], _c.c_int),
        "ac_get_state": ([_vp, ctypes.POINTER(_vp), ctypes.POINTER(_c.c_int),
                          ctypes.POINTER(_c.c_int), ctypes.POINTER(_c.c_int)], _c.c_int),
        "ac_closure_init": ([ctypes.POINTER(_vp), _c.c_int, _c.c_int, _c.c_int, _vp], _c.c_int),
        "ac_closure_quit": ([_vp], _c.c_int),
        "ac_closure_set_params": ([_vp, ctypes.POINTER(_c.c_float)], _c.c_int),
        "ac_closure_get_params": ([_vp, ctypes.POINTER(_c.c_float)], _c.c_int),
        "ac_closure_get_grads": ([_vp, ctypes.POINTER(_c.c_float)], _c.c_int),
        "ac_closure_set_scales": ([_vp, ctypes.POINTER(_c.c_float), ctypes.POINTER(_c.c_float)],
                                  _c.c_int),
        "ac_closure_forward": ([_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp)], _c.c_int),
        "ac_closure_forward_timings": ([_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                        ctypes.POINTER(_c.c_float)], _c.c_int),
        "ac_closure_backward": ([_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _pd], _c.c_int),
        "ac_closure_adam_step": ([_vp, _c.c_float, _c.c_float, _c.c_float, _c.c_float], _c.c_int),
        "ac_closure_apply": ([_vp, _vp, _c.c_double, ctypes.POINTER(_c.c_int)], _c.c_int),
        "ac_closure_launch_count": ([_vp, ctypes.POINTER(_c.c_ulonglong)], _c.c_int),
        "ac_closure_set_conv_path": ([_vp, _c.c_int], _c.c_int),
        "ac_diag_wait_timeout": ([_c.c_uint, _vp], _c.c_int),
        "ac_diag_exp_table": ([_vp, _c.c_longlong, _vp, _vp], _c.c_int),
        "ac_bounds_check_take": ([ctypes.POINTER(_c.c_ulonglong)], _c.c_int),
        "ac_bounds_check_selftest": ([ctypes.POINTER(_c.c_longlong)], _c.c_int),
        "ac_closure_get_conv_path": ([_vp, ctypes.POINTER(_c.c_int)], _c.c_int),
        "ac_closure_status": ([_vp], _c.c_int),
        "ac_restrict": ([ctypes.POINTER(_vp), _c.c_int, _c.c_int, _c.c_int, _c.c_int,
                         ctypes.POINTER(_vp), _vp], _c.c_int),
        "ac_strerror": ([_c.c_int], _c.c_char_p),
        "ac_last_cuda_error": ([], _c.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def _check(rc, where, value=None):
    if rc != AC_OK:
        raise AcError(rc, where, value)


def ac_strerror(code):
    return load_library().ac_strerror(code).decode()


def ac_last_cuda_error():
    return load_library().ac_last_cuda_error().decode()


def make_grid(n, L=(2 * math.pi,) * 3, layout=AC_LAYOUT_PERIODIC):
    return ac_grid(int(n[0]), int(n[1]), int(n[2]), float(L[0]), float(L[1]), float(L[2]),
                   int(layout))


def make_params(nu=5e-3, eta=5e-3, cs0=1.0, gamma=5.0 / 3.0, cp=1.0, lnrho0=0.0,
                force_amp=0.0, seed=0, precision=AC_FP64):
    return ac_params(nu, eta, cs0, gamma, cp, lnrho0, force_amp, seed, precision)


def ac_init(grid, params, stream=None):
    h = _vp()
    _check(load_library().ac_init(ctypes.byref(h), ctypes.byref(grid), ctypes.byref(params),
                                  _vp(stream or 0)), "ac_init")
    return h


def ac_quit(h):
    _check(load_library().ac_quit(h), "ac_quit")


def ac_set_stream(h, stream):
    _check(load_library().ac_set_stream(h, _vp(stream or 0)), "ac_set_stream")


def ac_bind_buffers(h, dev_ptrs):
    assert len(dev_ptrs) == 24
    arr = (_vp * 24)(*[int(p) for p in dev_ptrs])
    _check(load_library().ac_bind_buffers(h, arr), "ac_bind_buffers")


def ac_field_elems(h):
    n = ctypes.c_size_t()
    _check(load_library().ac_field_elems(h, ctypes.byref(n)), "ac_field_elems")
    return n.value


def _host_ptr(a, writable, elem=8):
    if isinstance(a, int):
        return a
    if hasattr(a, "data_ptr"):  # torch CPU tensor (e.g. pinned)
        assert a.dtype.is_floating_point and a.element_size() == elem and a.is_contiguous()
        return a.data_ptr()
    assert isinstance(a, np.ndarray) and a.dtype == (np.float64 if elem == 8 else np.float32)
    assert a.flags.c_contiguous and (a.flags.writeable or not writable)
    return a.ctypes.data


def ac_load_f32(h, field, host_src):
    """ac_load from float32 host memory (numpy float32 or a torch float32 CPU tensor)."""
    _check(load_library().ac_load_f32(h, field, _host_ptr(host_src, False, 4)), "ac_load_f32")


def ac_store_f32(h, field, host_dst):
    _check(load_library().ac_store_f32(h, field, _host_ptr(host_dst, True, 4)), "ac_store_f32")


def ac_load(h, field, host_src):
    _check(load_library().ac_load(h, field, _host_ptr(host_src, False)), "ac_load")


def ac_store(h, field, host_dst):
    _check(load_library().ac_store(h, field, _host_ptr(host_dst, True)), "ac_store")


def ac_load_w(h, field, host_src):
    _check(load_library().ac_load_w(h, field, _host_ptr(host_src, False)), "ac_load_w")


def ac_store_w(h, field, host_dst):
    _check(load_library().ac_store_w(h, field, _host_ptr(host_dst, True)), "ac_store_w")


def ac_integrate_substep(h, dt, s):
    _check(load_library().ac_integrate_substep(h, float(dt), int(s)), "ac_integrate_substep")


def ac_integrate_step(h, dt):
    _check(load_library().ac_integrate_step(h, float(dt)), "ac_integrate_step")


def ac_set_stencil_mode(h, mode):
    _check(load_library().ac_set_stencil_mode(h, int(mode)), "ac_set_stencil_mode")


def ac_get_stencil_path(h):
    fixed = ctypes.c_int()
    _check(load_library().ac_get_stencil_path(h, ctypes.byref(fixed)), "ac_get_stencil_path")
    return bool(fixed.value)


def ac_get_stencil_modes(h):
    """Substeps the integer-sum path ran with group scales, per-field scales and
    plain binary64 stencils (AC_STENCIL_MODE_GROUP/FIELD/PLAIN), as a 3-tuple."""
    out = (ctypes.c_ulonglong * 3)()
    _check(_lib.ac_get_stencil_modes(h, out), "ac_get_stencil_modes")
    return tuple(int(v) for v in out)


def ac_diag_fma_rate(precision, stream=None):
    """Fused multiply-adds per second of the library's FMA-chain probe kernel
    (AC_FP64: FP64 pipe, AC_FP32: FP32 pipes) on the current device."""
    out = ctypes.c_double()
    _check(_lib.ac_diag_fma_rate(precision, ctypes.byref(out), stream), "ac_diag_fma_rate")
    return out.value


def ac_set_kernel_timing(h, on):
    _check(_lib.ac_set_kernel_timing(h, 1 if on else 0), "ac_set_kernel_timing")


def ac_kernel_timings(h):
    """(prep_ms[3], kernel_ms[3], count[3]) per substep index since timing was
    switched on or last read."""
    a, b, c = (ctypes.c_double * 3)(), (ctypes.c_double * 3)(), (ctypes.c_int * 3)()
    _check(_lib.ac_kernel_timings(h, a, b, c), "ac_kernel_timings")
    return list(a), list(b), list(c)


def ac_last_cfl(h):
    out = ctypes.c_double()
    rc = load_library().ac_last_cfl(h, ctypes.byref(out))
    _check(rc, "ac_last_cfl", out.value)
    return out.value


def ac_periodic_halo(h):
    _check(load_library().ac_periodic_halo(h), "ac_periodic_halo")


def ac_reduce(h, op, quantity):
    out = ctypes.c_double()
    rc = load_library().ac_reduce(h, int(op), int(quantity), ctypes.byref(out))
    _check(rc, "ac_reduce", out.value)
    return out.value


def ac_reduce_noalloc(field_ptrs, grid, params, op, quantity, stream=None):
    """Reduction over caller-held device arrays without any device allocation
    (see include/ac.h); returns the value, raises AcError (with .value) on a
    non-finite input."""
    assert len(field_ptrs) == 8
    arr = (_vp * 8)(*[int(p) for p in field_ptrs])
    out = ctypes.c_double()
    rc = load_library().ac_reduce_noalloc(arr, ctypes.byref(grid), ctypes.byref(params), int(op),
                                          int(quantity), ctypes.byref(out), _vp(stream or 0))
    _check(rc, "ac_reduce_noalloc", out.value)
    return out.value


def ac_forcing_draw(seed, step):
    k = (ctypes.c_int * 3)()
    e = (ctypes.c_double * 3)()
    phi = ctypes.c_double()
    _check(load_library().ac_forcing_draw(seed & (2 ** 64 - 1), step, k, e, ctypes.byref(phi)),
           "ac_forcing_draw")
    return tuple(k), tuple(e), phi.value


def ac_set_forcing(h, k, e, phi):
    if k is None:
        _check(load_library().ac_set_forcing(h, None, None, 0.0), "ac_set_forcing")
        return
    kk = (ctypes.c_int * 3)(*[int(v) for v in k])
    ee = (ctypes.c_double * 3)(*[float(v) for v in e])
    _check(load_library().ac_set_forcing(h, kk, ee, float(phi)), "ac_set_forcing")


def ac_set_entropy_terms(h, K=0.0, zeta=0.0, heat=0.0, cool=0.0):
    _check(load_library().ac_set_entropy_terms(h, float(K), float(zeta), float(heat), float(cool)),
           "ac_set_entropy_terms")


def ac_set_stencil_order(h, order):
    _check(load_library().ac_set_stencil_order(h, int(order)), "ac_set_stencil_order")


def ac_get_stencil_order(h):
    o = ctypes.c_int()
    _check(load_library().ac_get_stencil_order(h, ctypes.byref(o)), "ac_get_stencil_order")
    return o.value


def ac_get_step(h):
    st = ctypes.c_ulonglong()
    ns = ctypes.c_int()
    _check(load_library().ac_get_step(h, ctypes.byref(st), ctypes.byref(ns)), "ac_get_step")
    return st.value, ns.value


def ac_set_step(h, step, next_substep=0):
    _check(load_library().ac_set_step(h, int(step), int(next_substep)), "ac_set_step")


def ac_launch_count(h):
    n = ctypes.c_ulonglong()
    _check(load_library().ac_launch_count(h, ctypes.byref(n)), "ac_launch_count")
    return n.value


def ac_get_state(h):
    ptrs = (_vp * 8)()
    prec, layout = ctypes.c_int(), ctypes.c_int()
    n = (ctypes.c_int * 3)()
    _check(load_library().ac_get_state(h, ptrs, ctypes.byref(prec), ctypes.byref(layout), n),
           "ac_get_state")
    return [p or 0 for p in ptrs], prec.value, layout.value, tuple(n)


# ---- learned closure -----------------------------------------------------------

AC_CLOSURE_NPARAMS = 41544


def _ptr8(ptrs):
    assert len(ptrs) == 8
    return (_vp * 8)(*[int(p) for p in ptrs])


def _f32(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def ac_restrict(fine_ptrs, fine_precision, n_fine, coarse_ptrs, stream=None):
    _check(load_library().ac_restrict(_ptr8(fine_ptrs), int(fine_precision), int(n_fine[0]),
                                      int(n_fine[1]), int(n_fine[2]), _ptr8(coarse_ptrs),
                                      _vp(stream or 0)), "ac_restrict")


def ac_closure_init(n, stream=None):
    c = _vp()
    _check(load_library().ac_closure_init(ctypes.byref(c), int(n[0]), int(n[1]), int(n[2]),
                                          _vp(stream or 0)), "ac_closure_init")
    return c


def ac_closure_quit(c):
    _check(load_library().ac_closure_quit(c), "ac_closure_quit")


def ac_closure_set_params(c, params):
    a, p = _f32(params)
    assert a.size == AC_CLOSURE_NPARAMS
    _check(load_library().ac_closure_set_params(c, p), "ac_closure_set_params")


def ac_closure_get_params(c):
    a = np.empty(AC_CLOSURE_NPARAMS, dtype=np.float32)
    _check(load_library().ac_closure_get_params(c, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
           "ac_closure_get_params")
    return a


def ac_closure_get_grads(c):
    a = np.empty(AC_CLOSURE_NPARAMS, dtype=np.float32)
    _check(load_library().ac_closure_get_grads(c, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
           "ac_closure_get_grads")
    return a


def ac_closure_set_scales(c, in_scale, out_scale):
    a, pa = _f32(in_scale)
    b, pb = _f32(out_scale)
    _check(load_library().ac_closure_set_scales(c, pa, pb), "ac_closure_set_scales")


def ac_closure_forward(c, in_ptrs, out_ptrs=None):
    _check(load_library().ac_closure_forward(c, _ptr8(in_ptrs),
                                             _ptr8(out_ptrs) if out_ptrs is not None else None),
           "ac_closure_forward")


def ac_closure_forward_timings(c, in_ptrs, out_ptrs):
    """Forward into out_ptrs; returns the device ms of its five launches
    (input pack, conv layers 1-3, output scale)."""
    ms = (ctypes.c_float * 5)()
    _check(load_library().ac_closure_forward_timings(c, _ptr8(in_ptrs), _ptr8(out_ptrs), ms),
           "ac_closure_forward_timings")
    return list(ms)


def ac_closure_backward(c, in_ptrs, target_ptrs):
    loss = ctypes.c_double()
    rc = load_library().ac_closure_backward(c, _ptr8(in_ptrs), _ptr8(target_ptrs),
                                            ctypes.byref(loss))
    _check(rc, "ac_closure_backward", loss.value)
    return loss.value


def ac_closure_adam_step(c, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    _check(load_library().ac_closure_adam_step(c, float(lr), float(beta1), float(beta2), float(eps)),
           "ac_closure_adam_step")


def ac_closure_apply(c, h, limit):
    applied = ctypes.c_int()
    _check(load_library().ac_closure_apply(c, h, float(limit), ctypes.byref(applied)),
           "ac_closure_apply")
    return bool(applied.value)


def ac_closure_launch_count(c):
    n = ctypes.c_ulonglong()
    _check(load_library().ac_closure_launch_count(c, ctypes.byref(n)), "ac_closure_launch_count")
    return n.value


def ac_diag_wait_timeout(polls, stream=None):
    """Run the bounded-wait diagnostic; returns the library's status code
    (AC_ERR_TIMEOUT is the expected outcome)."""
    return load_library().ac_diag_wait_timeout(int(polls), stream)


def ac_diag_exp_table(x, y, stream=None):
    """Table-driven exp diagnostic on device tensors: `x` (n binary64 values),
    `y` (4 n binary64 values, written); returns the library's status code."""
    return load_library().ac_diag_exp_table(_vp(x.data_ptr()), int(x.numel()),
                                            _vp(y.data_ptr()), stream)


def ac_bounds_check_take():
    """(status, first recorded word) of the global-index checks; status is
    AC_ERR_STATE for a library built without them."""
    w = _c.c_ulonglong(0)
    rc = load_library().ac_bounds_check_take(ctypes.byref(w))
    return rc, w.value


def ac_bounds_check_selftest():
    """(status, [index -5 checked, index 3 checked]) of the checked build."""
    out = (_c.c_longlong * 2)()
    rc = load_library().ac_bounds_check_selftest(out)
    return rc, [out[0], out[1]]


def ac_closure_set_conv_path(c, path):
    _check(load_library().ac_closure_set_conv_path(c, int(path)), "ac_closure_set_conv_path")


def ac_closure_get_conv_path(c):
    p = ctypes.c_int()
    _check(load_library().ac_closure_get_conv_path(c, ctypes.byref(p)), "ac_closure_get_conv_path")
    return p.value


def ac_closure_status(c):
    _check(load_library().ac_closure_status(c), "ac_closure_status")


# ---- batched ensemble --------------------------------------------------------

def ac_batch_init(boxes, common, stream=None):
    arr = (ac_box * len(boxes))(*boxes)
    b = _vp()
    _check(load_library().ac_batch_init(ctypes.byref(b), len(boxes), arr, ctypes.byref(common),
                                        _vp(stream or 0)), "ac_batch_init")
    return b


def ac_batch_quit(b):
    _check(load_library().ac_batch_quit(b), "ac_batch_quit")


def ac_batch_load(b, box, field, host_src):
    _check(load_library().ac_batch_load(b, box, field, _host_ptr(host_src, False)), "ac_batch_load")


def ac_batch_store(b, box, field, host_dst):
    _check(load_library().ac_batch_store(b, box, field, _host_ptr(host_dst, True)), "ac_batch_store")


def ac_batch_load_w(b, box, field, host_src):
    _check(load_library().ac_batch_load_w(b, box, field, _host_ptr(host_src, False)),
           "ac_batch_load_w")


def ac_batch_store_w(b, box, field, host_dst):
    _check(load_library().ac_batch_store_w(b, box, field, _host_ptr(host_dst, True)),
           "ac_batch_store_w")


def ac_batch_load_f32(b, box, field, host_src):
    _check(load_library().ac_batch_load_f32(b, box, field, _host_ptr(host_src, False, 4)),
           "ac_batch_load_f32")


def ac_batch_store_f32(b, box, field, host_dst):
    _check(load_library().ac_batch_store_f32(b, box, field, _host_ptr(host_dst, True, 4)),
           "ac_batch_store_f32")


def ac_batch_integrate_substep(b, dt, s):
    _check(load_library().ac_batch_integrate_substep(b, float(dt), int(s)),
           "ac_batch_integrate_substep")


def ac_batch_integrate_step(b, dt):
    _check(load_library().ac_batch_integrate_step(b, float(dt)), "ac_batch_integrate_step")


def ac_batch_set_graph(b, enable):
    _check(load_library().ac_batch_set_graph(b, int(bool(enable))), "ac_batch_set_graph")


def ac_batch_tune(b, dt, cache_path=None):
    zc = ctypes.c_int()
    cp = cache_path.encode() if cache_path else None
    _check(load_library().ac_batch_tune(b, float(dt), cp, ctypes.byref(zc)), "ac_batch_tune")
    return zc.value


def ac_batch_set_tiling(b, zc, shapes=None):
    arr = None
    if shapes is not None:
        arr = (ctypes.c_int * len(shapes))(*[int(v) for v in shapes])
    _check(load_library().ac_batch_set_tiling(b, int(zc), arr), "ac_batch_set_tiling")


def ac_batch_get_tiling(b, nbox):
    """(z extent, list of nbox tile shapes, [ms of the default split, ms tuned])."""
    zc = ctypes.c_int()
    arr = (ctypes.c_int * nbox)()
    ms = (ctypes.c_float * 2)()
    _check(load_library().ac_batch_get_tiling(b, ctypes.byref(zc), arr, ms), "ac_batch_get_tiling")
    return zc.value, list(arr), [ms[0], ms[1]]


def ac_batch_reduce(b, box, op, quantity):
    out = ctypes.c_double()
    rc = load_library().ac_batch_reduce(b, box, int(op), int(quantity), ctypes.byref(out))
    _check(rc, "ac_batch_reduce", out.value)
    return out.value


def ac_batch_info(b):
    cells = ctypes.c_longlong()
    items, zc, ctas = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    launches = ctypes.c_ulonglong()
    _check(load_library().ac_batch_info(b, ctypes.byref(cells), ctypes.byref(items),
                                        ctypes.byref(zc), ctypes.byref(ctas),
                                        ctypes.byref(launches)), "ac_batch_info")
    return dict(cells=cells.value, items=items.value, zc=zc.value, ctas=ctas.value,
                launches=launches.value)


def _int3(v):
    return (ctypes.c_int * 3)(*[int(x) for x in v])


def ac_decomp_partition(count):
    p = (ctypes.c_int * 3)()
    _check(load_library().ac_decomp_partition(int(count), p), "ac_decomp_partition")
    return tuple(p)


def ac_decomp_coord(p, rank):
    c = (ctypes.c_int * 3)()
    _check(load_library().ac_decomp_coord(_int3(p), int(rank), c), "ac_decomp_coord")
    return tuple(c)


def ac_decomp_segment(nloc, seg):
    """(dir, src_b0, dst_b0, ext) of halo segment `seg` (0..17), padded coordinates."""
    out = [(ctypes.c_int * 3)() for _ in range(4)]
    _check(load_library().ac_decomp_segment(_int3(nloc), int(seg), *out), "ac_decomp_segment")
    return tuple(tuple(v) for v in out)


def ac_decomp_init(grid, params, p, stream=None):
    d = _vp()
    _check(load_library().ac_decomp_init(ctypes.byref(d), ctypes.byref(grid),
                                         ctypes.byref(params), _int3(p), stream),
           "ac_decomp_init")
    return d


def ac_decomp_info(d):
    p, nl = (ctypes.c_int * 3)(), (ctypes.c_int * 3)()
    m, la = ctypes.c_int(), ctypes.c_ulonglong()
    _check(load_library().ac_decomp_info(d, p, nl, ctypes.byref(m), ctypes.byref(la)),
           "ac_decomp_info")
    return dict(p=tuple(p), nloc=tuple(nl), messages=m.value, launches=la.value)


class Decomp:
    """A periodic grid split into p = (px, py, pz) subdomains with halo exchange
    (all subdomains on the current device)."""

    def __init__(self, n, p, L=(2 * math.pi,) * 3, precision=AC_FP64, nu=5e-3, eta=5e-3,
                 cs0=1.0, gamma=5.0 / 3.0, cp=1.0, lnrho0=0.0, force_amp=0.0, seed=0,
                 stream=None, overlap=True):
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        self.n = tuple(n)
        self.d = ac_decomp_init(make_grid(n, L),
                                make_params(nu, eta, cs0, gamma, cp, lnrho0, force_amp, seed,
                                            precision), p, stream)
        _check(_lib.ac_decomp_set_overlap(self.d, 1 if overlap else 0), "ac_decomp_set_overlap")
        self._closed = False

    def set_overlap(self, on):
        _check(_lib.ac_decomp_set_overlap(self.d, 1 if on else 0), "ac_decomp_set_overlap")

    def _io(self, fn, arr, where):
        _check(fn(self.d, AC_ALL, arr.ctypes.data_as(_vp)), where)

    def load(self, f):
        self._io(_lib.ac_decomp_load, np.ascontiguousarray(f, dtype=np.float64), "ac_decomp_load")

    def load_w(self, w):
        self._io(_lib.ac_decomp_load_w, np.ascontiguousarray(w, dtype=np.float64),
                 "ac_decomp_load_w")

    def store(self):
        nx, ny, nz = self.n
        out = np.empty((8, nz, ny, nx))
        self._io(_lib.ac_decomp_store, out, "ac_decomp_store")
        return out

    def store_w(self):
        nx, ny, nz = self.n
        out = np.empty((8, nz, ny, nx))
        self._io(_lib.ac_decomp_store_w, out, "ac_decomp_store_w")
        return out

    def substep(self, dt, s):
        _check(_lib.ac_decomp_integrate_substep(self.d, float(dt), int(s)),
               "ac_decomp_integrate_substep")

    def step(self, dt):
        _check(_lib.ac_decomp_integrate_step(self.d, float(dt)), "ac_decomp_integrate_step")

    def info(self):
        return ac_decomp_info(self.d)

    def close(self):
        if not self._closed:
            _lib.ac_decomp_quit(self.d)
            self._closed = True

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """An ensemble of boxes: `boxes` is a list of (n, L, nu, eta)."""

    def __init__(self, boxes, precision=AC_FP32, cs0=1.0, gamma=5.0 / 3.0, cp=1.0, lnrho0=0.0,
                 stream=None):
        self.specs = [(tuple(n), tuple(L), nu, eta) for n, L, nu, eta in boxes]
        arr = [ac_box(n[0], n[1], n[2], L[0], L[1], L[2], nu, eta) for n, L, nu, eta in self.specs]
        common = make_params(cs0=cs0, gamma=gamma, cp=cp, lnrho0=lnrho0, precision=precision)
        if stream is None:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        self.b = ac_batch_init(arr, common, stream)
        self._closed = False

    def load(self, box, f):
        ac_batch_load(self.b, box, AC_ALL, np.ascontiguousarray(f, dtype=np.float64))

    def store(self, box):
        nx, ny, nz = self.specs[box][0]
        out = np.empty((8, nz, ny, nx))
        ac_batch_store(self.b, box, AC_ALL, out)
        return out

    def store_w(self, box):
        nx, ny, nz = self.specs[box][0]
        out = np.empty((8, nz, ny, nx))
        ac_batch_store_w(self.b, box, AC_ALL, out)
        return out

    def step(self, dt):
        ac_batch_integrate_step(self.b, dt)

    def substep(self, dt, s):
        ac_batch_integrate_substep(self.b, dt, s)

    def close(self):
        if not self._closed:
            ac_batch_quit(self.b)
            self._closed = True

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Simulation:
    """A handle whose state lives in torch-owned device tensors.

    ``state[b]`` (b = 0, 1) are the two alternating (8, elems) state buffers
    and ``w`` the (8, elems) accumulator; the library's current state is
    ``state[current]``.  Rows are padded to 16-byte multiples.
    """

    def __init__(self, n, L=(2 * math.pi,) * 3, layout=AC_LAYOUT_PERIODIC, precision=AC_FP64,
                 nu=5e-3, eta=5e-3, cs0=1.0, gamma=5.0 / 3.0, cp=1.0, lnrho0=0.0,
                 force_amp=0.0, seed=0, device="cuda", stream=None, order=6, K=0.0, zeta=0.0,
                 heat=0.0, cool=0.0):
        import torch
        self.n = tuple(n)
        self.precision = precision
        self.layout = layout
        if stream is None:
            stream = torch.cuda.current_stream(device).cuda_stream
        self.h = ac_init(make_grid(n, L, layout),
                         make_params(nu, eta, cs0, gamma, cp, lnrho0, force_amp, seed, precision),
                         stream)
        self.elems = ac_field_elems(self.h)
        fdt = torch.float64 if precision == AC_FP64 else torch.float32
        wdt = torch.float32 if precision == AC_FP32 else torch.float64
        row = (self.elems + 3) // 4 * 4
        self.state = torch.zeros((2, 8, row), dtype=fdt, device=device)
        self.w = torch.zeros((8, row), dtype=wdt, device=device)
        ptrs = [self.state[b, q].data_ptr() for b in range(2) for q in range(8)]
        ptrs += [self.w[q].data_ptr() for q in range(8)]
        ac_bind_buffers(self.h, ptrs)
        if order != 6:
            ac_set_stencil_order(self.h, order)
        if K or zeta or heat or cool:
            ac_set_entropy_terms(self.h, K, zeta, heat, cool)
        self._closed = False

    def load(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        ac_load(self.h, AC_ALL, f)

    def store(self):
        nx, ny, nz = self.n
        out = np.empty((8, nz, ny, nx))
        ac_store(self.h, AC_ALL, out)
        return out

    def load_w(self, w):
        ac_load_w(self.h, AC_ALL, np.ascontiguousarray(w, dtype=np.float64))

    def store_w(self):
        nx, ny, nz = self.n
        out = np.empty((8, nz, ny, nx))
        ac_store_w(self.h, AC_ALL, out)
        return out

    def substep(self, dt, s):
        ac_integrate_substep(self.h, dt, s)

    def step(self, dt):
        ac_integrate_step(self.h, dt)

    def reduce(self, op, quantity):
        return ac_reduce(self.h, op, quantity)

    def close(self):
        if not self._closed:
            ac_quit(self.h)
            self._closed = True

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

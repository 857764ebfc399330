"""ctypes binding of libcncpd (include/cncpd.h): the C entry points under
the same names, with argument marshalling only.  Loading fails loudly when
the library has not been built; there is no fallback implementation."""

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libcncpd.so")

CNCPD_F64, CNCPD_F32, CNCPD_BF16, CNCPD_BF16X2 = 0, 1, 2, 3
CNCPD_OK = 0
ERRORS = {-1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ENONFINITE", -5: "ETIMEOUT",
          -6: "ESTATE", -7: "ESINGULAR"}


class cncpd_opts(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("max_it", ctypes.c_int),
                ("lra_eps", ctypes.c_double), ("lra_max_it", ctypes.c_int),
                ("delta_w", ctypes.c_double), ("use_core", ctypes.c_int),
                ("reupdate", ctypes.c_int), ("storage", ctypes.c_int),
                ("use_graph", ctypes.c_int), ("profile", ctypes.c_int),
                ("tensor_cores", ctypes.c_int), ("autotune", ctypes.c_int), ("tf32", ctypes.c_int),
                ("stream_x", ctypes.c_int), ("reserved", ctypes.c_int * 2)]


class cncpd_stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("total_iters", ctypes.c_int),
                ("reupdates", ctypes.c_int), ("converged", ctypes.c_int),
                ("F", ctypes.c_double), ("relerr", ctypes.c_double), ("fit", ctypes.c_double),
                ("seconds", ctypes.c_double), ("x_bytes", ctypes.c_double),
                ("stream_ms", ctypes.c_double), ("stream_launches", ctypes.c_int),
                ("lra_sweeps", ctypes.c_int), ("lra_relerr", ctypes.c_double),
                ("trail_ms", ctypes.c_double), ("lead_ms", ctypes.c_double),
                ("launches", ctypes.c_longlong), ("lead_plan", ctypes.c_int),
                ("lead_plan_tuned", ctypes.c_int), ("trail_ranges", ctypes.c_int),
                ("trail_tensor_cores", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class CncpdError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_PP = ctypes.POINTER(ctypes.c_void_p)

SIGNATURES = {
    "cncpd_default_opts": (None, [ctypes.POINTER(cncpd_opts)]),
    "cncpd_create": (_I, [ctypes.POINTER(_P), _I, _I, ctypes.POINTER(ctypes.c_int64), _PP, _I,
                          ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_ubyte),
                          ctypes.POINTER(cncpd_opts), _P]),
    "cncpd_set_factors": (_I, [_P, _I, _I, _P, _I]),
    "cncpd_set_factors_all": (_I, [_P, _P, _I]),
    "cncpd_set_core": (_I, [_P, _I, ctypes.POINTER(_D)]),
    "cncpd_lra": (_I, [_P, ctypes.POINTER(_I), _PP, _I, ctypes.POINTER(cncpd_stats)]),
    "cncpd_step": (_I, [_P, _I, ctypes.POINTER(cncpd_stats)]),
    "cncpd_fit": (_I, [_P, ctypes.POINTER(cncpd_stats)]),
    "cncpd_factors": (_I, [_P, _I, _I, _P, _I]),
    "cncpd_core": (_I, [_P, _I, ctypes.POINTER(_D)]),
    "cncpd_lra_factors": (_I, [_P, _I, _I, _P, _I]),
    "cncpd_global_fit": (_I, [_P, ctypes.POINTER(_D)]),
    "cncpd_objective_grad": (_I, [_P, ctypes.POINTER(_D), _PP, _PP, _I]),
    "cncpd_objective_grad_at": (_I, [_P, _PP, _I, ctypes.POINTER(_D), _PP, _PP, _I]),
    "cncpd_mttkrp": (_I, [_P, _I, _I, _P, _I]),
    "cncpd_lipschitz": (_I, [ctypes.POINTER(_D), _I, ctypes.POINTER(_D)]),
    "cncpd_save_state": (_I, [_P, ctypes.POINTER(_P), ctypes.POINTER(ctypes.c_size_t)]),
    "cncpd_load_state": (_I, [_P, _P, ctypes.c_size_t]),
    "cncpd_free_blob": (None, [_P]),
    "cncpd_mttkrp_last_mode_noalloc": (_I, [_P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, _P, _P,
                                            _I, _P, _P]),
    "cncpd_check_wait_timeout": (_I, [_P, _D]),
    "cncpd_destroy": (None, [_P]),
    "cncpd_last_error": (ctypes.c_char_p, []),
}

_lib = None


def lib():
    """The loaded library (raises if it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def check(code):
    if code != CNCPD_OK:
        raise CncpdError(code, lib().cncpd_last_error().decode())
    return code


def _wrap(name):
    def call(*args):
        return getattr(lib(), name)(*args)
    call.__name__ = name
    return call


for _name in SIGNATURES:
    globals()[_name] = _wrap(_name)

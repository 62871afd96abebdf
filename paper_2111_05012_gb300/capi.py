"""ctypes binding of the C ABI in include/lqcd_amg.h.

Argument marshalling only: every function here forwards to the entry point of
the same name in libamg.so and turns a non-zero status into AMGError.  Device
vectors are passed as torch tensors (or raw integer device pointers); streams
as torch.cuda.Stream objects, raw handles or None (the default stream).
There is no fallback: if the library is missing the import of a function
fails loudly.
"""
import ctypes
import os

import numpy as np

from .build import LIB

AMG_OK, AMG_EINVAL, AMG_ENOMEM, AMG_ECUDA, AMG_NOT_CONVERGED, AMG_NAN, AMG_TIMEOUT, AMG_EIO = range(8)
AMG_F64, AMG_F32, AMG_F16, AMG_BF16, AMG_F64X, AMG_F64D = range(6)
AMG_MAX_LEVELS = 4

STATUS_NAMES = {0: "AMG_OK", 1: "AMG_EINVAL", 2: "AMG_ENOMEM", 3: "AMG_ECUDA", 4: "AMG_NOT_CONVERGED",
                5: "AMG_NAN", 6: "AMG_TIMEOUT", 7: "AMG_EIO"}


class AMGError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class amg_params(ctypes.Structure):
    _fields_ = [
        ("nlevels", ctypes.c_int),
        ("block", (ctypes.c_int * 4) * (AMG_MAX_LEVELS - 1)),
        ("nvec", ctypes.c_int * (AMG_MAX_LEVELS - 1)),
        ("n_init", ctypes.c_int),
        ("n_adapt", ctypes.c_int),
        ("sap_iters", ctypes.c_int),
        ("mr_iters", ctypes.c_int),
        ("coarse_tol", ctypes.c_double),
        ("coarse_maxit", ctypes.c_int),
        ("coarse_ell", ctypes.c_int),
        ("inter_m", ctypes.c_int),
        ("inter_tol", ctypes.c_double),
        ("inter_maxit", ctypes.c_int),
        ("outer_m", ctypes.c_int),
        ("prec_smoother", ctypes.c_int),
        ("prec_coarse", ctypes.c_int),
        ("prec_coarsest", ctypes.c_int),
        ("sap_variant", ctypes.c_int),
        ("outer_solver", ctypes.c_int),
        ("prec_vectors", ctypes.c_int),
        ("mbicgs_tol", ctypes.c_double),
        ("mbicgs_maxit", ctypes.c_int),
        ("sap_eo", ctypes.c_int),
        ("coarse_tc", ctypes.c_int),
        ("resid_pair", ctypes.c_int),
    ]


class amg_solve_info(ctypes.Structure):
    _fields_ = [
        ("iters", ctypes.c_int),
        ("restarts", ctypes.c_int),
        ("converged", ctypes.c_int),
        ("true_rel_residual", ctypes.c_double),
        ("ms_total", ctypes.c_double),
        ("ms_coarse", ctypes.c_double),
        ("ms_smoother", ctypes.c_double),
        ("ms_restrict_prolong", ctypes.c_double),
        ("ms_other", ctypes.c_double),
        ("coarse_cycles", ctypes.c_int),
        ("used_nn", ctypes.c_int),
        ("nn_fallback", ctypes.c_int),
        ("cycles", ctypes.c_int),
        ("ms_products", ctypes.c_double),
        ("ms_orthogonalisation", ctypes.c_double),
        ("ms_true_residual", ctypes.c_double),
        ("batch_width", ctypes.c_int),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class amg_train_params(ctypes.Structure):
    _fields_ = [("npairs", ctypes.c_int), ("batch", ctypes.c_int), ("lr", ctypes.c_double),
                ("seed", ctypes.c_uint64)]


_vp = ctypes.c_void_p
_ip = ctypes.POINTER(ctypes.c_int)
_dp = ctypes.POINTER(ctypes.c_double)
_i = ctypes.c_int
_d = ctypes.c_double

# name -> (restype, argtypes); the list mirrors include/lqcd_amg.h
PROTOTYPES = {
    "amg_last_error": (ctypes.c_char_p, []),
    "amg_launch_count": (ctypes.c_ulonglong, []),
    "amg_params_default": (None, [ctypes.POINTER(amg_params)]),
    "amg_lattice_create": (_i, [_ip, _i, ctypes.POINTER(_vp)]),
    "amg_lattice_destroy": (None, [_vp]),
    "amg_gauge_create": (_i, [_vp, _dp, ctypes.POINTER(_vp)]),
    "amg_gauge_destroy": (None, [_vp]),
    "amg_gauge_random": (_i, [_vp, _d, ctypes.c_uint64, ctypes.POINTER(_vp)]),
    "amg_gauge_get": (_i, [_vp, _dp]),
    "amg_random_normal": (_i, [ctypes.c_uint64, _i, ctypes.c_uint64, ctypes.c_uint64, _vp, _vp]),
    "amg_dirac_create": (_i, [_vp, _d, _d, ctypes.POINTER(_vp)]),
    "amg_dirac_destroy": (None, [_vp]),
    "amg_dirac_get_clover": (_i, [_vp, _dp]),
    "amg_apply_D": (_i, [_vp, _vp, _vp, _i, _i, _vp]),
    "amg_apply_D_noalloc": (_i, [_vp, _vp, _vp, _i, _i, _vp]),
    "amg_apply_Dsap": (_i, [_vp, _ip, _vp, _vp, _i, _i, _vp]),
    "amg_dirac_time": (_i, [_vp, _vp, _i, _i, _i, _vp, ctypes.POINTER(ctypes.c_float)]),
    "amg_coarse_time": (_i, [_vp, _i, _vp, _i, _i, _i, _vp, ctypes.POINTER(ctypes.c_float)]),
    "amg_setup": (_i, [_vp, ctypes.POINTER(amg_params), ctypes.POINTER(_dp), ctypes.POINTER(_vp)]),
    "amg_setup_from_vectors": (_i, [_vp, ctypes.POINTER(amg_params), ctypes.POINTER(_dp), ctypes.POINTER(_vp)]),
    "amg_hierarchy_destroy": (None, [_vp]),
    "amg_level_info": (_i, [_vp, _i, _ip, _ip]),
    "amg_get_vectors": (_i, [_vp, _i, _dp]),
    "amg_get_coarse_op": (_i, [_vp, _i, _dp]),
    "amg_setup_save": (_i, [_vp, ctypes.c_char_p]),
    "amg_setup_load": (_i, [_vp, ctypes.c_char_p, ctypes.POINTER(_vp)]),
    "amg_apply_coarse": (_i, [_vp, _i, _vp, _vp, _i, _i, _vp]),
    "amg_restrict": (_i, [_vp, _i, _vp, _vp, _i, _i, _vp]),
    "amg_prolong": (_i, [_vp, _i, _vp, _vp, _i, _i, _vp]),
    "amg_sap": (_i, [_vp, _vp, _vp, _i, _i, _vp]),
    "amg_sap_coarse": (_i, [_vp, _i, _vp, _vp, _i, _i, _vp]),
    "amg_precondition": (_i, [_vp, _vp, _vp, _vp]),
    "amg_solve": (_i, [_vp, _vp, _vp, _i, _d, _i, _i, ctypes.POINTER(amg_solve_info), _vp]),
    "amg_solve_ragged": (_i, [ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp), _i, _d, _i,
                              ctypes.POINTER(amg_solve_info), _vp]),
    "amg_set_ragged_fusion": (None, [_i]),
    "amg_dirac_tune": (_i, [_vp, _i, _ip, _ip, _ip]),
    "amg_dirac_set_shape": (_i, [_i, _i, _i, _i]),
    "amg_nn_create": (_i, [_vp, _i, _ip, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(_vp)]),
    "amg_nn_destroy": (None, [_vp]),
    "amg_nn_get_weights": (_i, [_vp, _i, ctypes.POINTER(ctypes.c_float)]),
    "amg_nn_layer_forward": (_i, [_vp, _i, _vp, _vp, _vp]),
    "amg_nn_layer_backward": (_i, [_vp, _i, _vp, _vp, _vp, _dp, _vp]),
    "amg_nn_apply": (_i, [_vp, _vp, _vp, _vp]),
    "amg_nn_train_step": (_i, [_vp, _vp, _vp, _i, _d, _dp, _vp]),
    "amg_hierarchy_set_nn": (_i, [_vp, _vp]),
    "amg_train_params_default": (None, [ctypes.POINTER(amg_train_params)]),
    "amg_learned_train": (_i, [_vp, _vp, ctypes.POINTER(amg_train_params), _dp, _vp]),
}

_lib = None


def load():
    """Load libamg.so (built in-tree by __graft_entry__.build()); raises if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError(f"{LIB} is missing: build it with __graft_entry__.build()")
        lib = ctypes.CDLL(LIB)
        for name, (res, args) in PROTOTYPES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(st):
    if st != AMG_OK:
        raise AMGError(st, load().amg_last_error().decode())
    return st


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    raise TypeError(f"cannot pass {type(x)} as a device pointer")


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _host_f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def amg_last_error():
    return load().amg_last_error().decode()


def amg_launch_count():
    return int(load().amg_launch_count())


def amg_params_default():
    p = amg_params()
    load().amg_params_default(ctypes.byref(p))
    return p


def amg_lattice_create(dims, antiperiodic_t=True):
    h = _vp()
    _check(load().amg_lattice_create((ctypes.c_int * 4)(*dims), int(bool(antiperiodic_t)), ctypes.byref(h)))
    return h


def amg_lattice_destroy(h):
    load().amg_lattice_destroy(h)


def amg_gauge_create(lat, U):
    """U: float64 array [site][mu][3][3][re, im] (e.g. lqcd_inputs.to_interleaved of a gauge field)."""
    a, p = _host_f64(U)
    h = _vp()
    _check(load().amg_gauge_create(lat, p, ctypes.byref(h)))
    return h


def amg_gauge_destroy(h):
    load().amg_gauge_destroy(h)


def amg_gauge_random(lat, eps, seed):
    h = _vp()
    _check(load().amg_gauge_random(lat, float(eps), int(seed), ctypes.byref(h)))
    return h


def amg_gauge_get(g, volume):
    out = np.empty((volume, 4, 3, 3, 2), dtype=np.float64)
    _check(load().amg_gauge_get(g, out.ctypes.data_as(_dp)))
    return out


def amg_random_normal(seed, stream_id, start, count, out, stream=None):
    """Complex normals start..start+count-1 of (seed, stream_id) into the device tensor out (2*count doubles)."""
    _check(load().amg_random_normal(int(seed), int(stream_id), int(start), int(count), _ptr(out), _stream(stream)))


def amg_dirac_create(gauge, kappa, csw):
    h = _vp()
    _check(load().amg_dirac_create(gauge, float(kappa), float(csw), ctypes.byref(h)))
    return h


def amg_dirac_destroy(h):
    load().amg_dirac_destroy(h)


def amg_dirac_get_clover(d, volume):
    out = np.empty((volume, 2, 6, 6, 2), dtype=np.float64)
    _check(load().amg_dirac_get_clover(d, out.ctypes.data_as(_dp)))
    return out


def amg_apply_D(d, inp, out, nrhs=1, prec=AMG_F64, stream=None):
    _check(load().amg_apply_D(d, _ptr(inp), _ptr(out), int(nrhs), int(prec), _stream(stream)))


def amg_apply_D_noalloc(d, inp, out, nrhs=1, prec=AMG_F64, stream=None):
    _check(load().amg_apply_D_noalloc(d, _ptr(inp), _ptr(out), int(nrhs), int(prec), _stream(stream)))


def amg_dirac_tune(d, prec):
    """Autotune the stencil's launch shape for prec; returns (threads, per_sm, regs_ctas)."""
    a, b, m = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load().amg_dirac_tune(d, int(prec), ctypes.byref(a), ctypes.byref(b), ctypes.byref(m)))
    return a.value, b.value, m.value


def amg_dirac_set_shape(prec, threads, per_sm, regs_ctas=0):
    _check(load().amg_dirac_set_shape(int(prec), int(threads), int(per_sm), int(regs_ctas)))


def amg_dirac_time(d, inp, nrhs=1, prec=AMG_F32, reps=20, stream=None):
    """Mean milliseconds per application of D (internal layout, kernel only)."""
    ms = ctypes.c_float()
    _check(load().amg_dirac_time(d, _ptr(inp), int(nrhs), int(prec), int(reps), _stream(stream), ctypes.byref(ms)))
    return float(ms.value)


def amg_coarse_time(h, level, inp, nrhs=1, prec=AMG_F32, reps=20, stream=None):
    """Mean milliseconds per application of the coarse stencil (kernel only)."""
    ms = ctypes.c_float()
    _check(load().amg_coarse_time(h, int(level), _ptr(inp), int(nrhs), int(prec), int(reps), _stream(stream),
                                  ctypes.byref(ms)))
    return float(ms.value)


def amg_apply_Dsap(d, block, inp, out, nrhs=1, prec=AMG_F64, stream=None):
    _check(load().amg_apply_Dsap(d, (ctypes.c_int * 4)(*block), _ptr(inp), _ptr(out), int(nrhs), int(prec),
                                 _stream(stream)))


def _vec_list(vecs):
    """Pointer array of AMG_MAX_LEVELS entries (NULL past the given levels);
    each entry a host array (float64) or a float64 device tensor."""
    if len(vecs) > AMG_MAX_LEVELS:
        raise ValueError("more vector sets than levels")
    keep, ptrs = [], []
    for v in vecs:
        if hasattr(v, "data_ptr"):
            keep.append(v)
            ptrs.append(ctypes.cast(_ptr(v), _dp))
        else:
            a = np.ascontiguousarray(v, dtype=np.float64)
            keep.append(a)
            ptrs.append(a.ctypes.data_as(_dp))
    lst = (_dp * AMG_MAX_LEVELS)(*ptrs)
    return keep, lst


def amg_setup(d, params, init_vecs):
    """init_vecs: list (one per coarsening) of float64 arrays of canonical vectors."""
    keep, lst = _vec_list(init_vecs)
    h = _vp()
    _check(load().amg_setup(d, ctypes.byref(params), lst, ctypes.byref(h)))
    return h


def amg_setup_from_vectors(d, params, vecs):
    keep, lst = _vec_list(vecs)
    h = _vp()
    _check(load().amg_setup_from_vectors(d, ctypes.byref(params), lst, ctypes.byref(h)))
    return h


def amg_hierarchy_destroy(h):
    load().amg_hierarchy_destroy(h)


def amg_level_info(h, level):
    dims = (ctypes.c_int * 4)()
    nc = ctypes.c_int()
    _check(load().amg_level_info(h, int(level), dims, ctypes.byref(nc)))
    return tuple(dims), nc.value


def amg_get_vectors(h, coarsening, nvec, volume, ndof=12):
    out = np.empty((nvec, volume, ndof, 2), dtype=np.float64)
    _check(load().amg_get_vectors(h, int(coarsening), out.ctypes.data_as(_dp)))
    return out


def amg_get_coarse_op(h, level):
    dims, nc = amg_level_info(h, level)
    vc = int(np.prod(dims))
    out = np.empty((vc, 9, nc, nc, 2), dtype=np.float64)
    _check(load().amg_get_coarse_op(h, int(level), out.ctypes.data_as(_dp)))
    return out


def amg_setup_save(h, path):
    _check(load().amg_setup_save(h, str(path).encode()))


def amg_setup_load(d, path):
    h = _vp()
    _check(load().amg_setup_load(d, str(path).encode(), ctypes.byref(h)))
    return h


def amg_apply_coarse(h, level, inp, out, nrhs=1, prec=AMG_F64, stream=None):
    _check(load().amg_apply_coarse(h, int(level), _ptr(inp), _ptr(out), int(nrhs), int(prec), _stream(stream)))


def amg_restrict(h, coarsening, fine, coarse, nrhs=1, prec=AMG_F64, stream=None):
    _check(load().amg_restrict(h, int(coarsening), _ptr(fine), _ptr(coarse), int(nrhs), int(prec),
                               _stream(stream)))


def amg_prolong(h, coarsening, coarse, fine, nrhs=1, prec=AMG_F64, stream=None):
    _check(load().amg_prolong(h, int(coarsening), _ptr(coarse), _ptr(fine), int(nrhs), int(prec),
                              _stream(stream)))


def amg_sap(h, b, x, prec=AMG_F32, stream=None, nrhs=1):
    _check(load().amg_sap(h, _ptr(b), _ptr(x), int(nrhs), int(prec), _stream(stream)))


def amg_sap_coarse(h, level, b, x, nrhs=1, prec=AMG_F32, stream=None):
    _check(load().amg_sap_coarse(h, int(level), _ptr(b), _ptr(x), int(nrhs), int(prec), _stream(stream)))


def amg_precondition(h, b, x, stream=None):
    _check(load().amg_precondition(h, _ptr(b), _ptr(x), _stream(stream)))


def amg_solve(h, b, x, nrhs=1, tol=1e-10, maxit=500, use_x0=False, stream=None, raise_on_nonconv=True):
    """Returns (status, amg_solve_info)."""
    info = amg_solve_info()
    st = load().amg_solve(h, _ptr(b), _ptr(x), int(nrhs), float(tol), int(maxit), int(bool(use_x0)),
                          ctypes.byref(info), _stream(stream))
    if st != AMG_OK and (st != AMG_NOT_CONVERGED or raise_on_nonconv):
        _check(st)
    return st, info


def amg_set_ragged_fusion(on):
    load().amg_set_ragged_fusion(1 if on else 0)


def amg_solve_ragged(hs, bs, xs, tol=1e-10, maxit=500, stream=None, raise_on_nonconv=True):
    """Independent problems hs[i] (hierarchies), bs[i] / xs[i] device tensors.
    Returns (status, [amg_solve_info])."""
    n = len(hs)
    ha = (_vp * n)(*hs)
    ba = (_vp * n)(*[_ptr(b) for b in bs])
    xa = (_vp * n)(*[_ptr(x) for x in xs])
    infos = (amg_solve_info * n)()
    st = load().amg_solve_ragged(ha, ba, xa, n, float(tol), int(maxit), infos, _stream(stream))
    if st != AMG_OK and (st != AMG_NOT_CONVERGED or raise_on_nonconv):
        _check(st)
    return st, list(infos)


# ---- learned preconditioner ----

def nn_weight_sizes(channels):
    return [channels[l + 1] * channels[l] * 9 * 16 * 2 for l in range(len(channels) - 1)]


def amg_nn_create(d, channels, weights):
    """channels e.g. [1, 4, 1]; weights: flat float array (layer after layer)."""
    w = np.ascontiguousarray(weights, dtype=np.float32).reshape(-1)
    assert w.size == sum(nn_weight_sizes(channels))
    h = _vp()
    _check(load().amg_nn_create(d, len(channels) - 1, (ctypes.c_int * len(channels))(*channels),
                                w.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), ctypes.byref(h)))
    return h


def amg_nn_destroy(nn):
    load().amg_nn_destroy(nn)


def amg_nn_get_weights(nn, channels, effective=True):
    out = np.empty(sum(nn_weight_sizes(channels)), dtype=np.float32)
    _check(load().amg_nn_get_weights(nn, int(bool(effective)), out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
    return out


def amg_nn_layer_forward(nn, layer, inp, out, stream=None):
    _check(load().amg_nn_layer_forward(nn, int(layer), _ptr(inp), _ptr(out), _stream(stream)))


def amg_nn_layer_backward(nn, layer, inp, grad_out, grad_in=None, want_wgrad=True, wsize=None, stream=None):
    gw = np.zeros(wsize, dtype=np.float64) if want_wgrad else None
    _check(load().amg_nn_layer_backward(nn, int(layer), _ptr(inp), _ptr(grad_out), _ptr(grad_in),
                                        gw.ctypes.data_as(_dp) if gw is not None else None, _stream(stream)))
    return gw


def amg_nn_apply(nn, inp, out, stream=None):
    _check(load().amg_nn_apply(nn, _ptr(inp), _ptr(out), _stream(stream)))


def amg_nn_train_step(nn, r, e, npairs, lr=1e-3, stream=None):
    loss = ctypes.c_double()
    _check(load().amg_nn_train_step(nn, _ptr(r), _ptr(e), int(npairs), float(lr), ctypes.byref(loss),
                                    _stream(stream)))
    return loss.value


def amg_hierarchy_set_nn(h, nn):
    _check(load().amg_hierarchy_set_nn(h, nn))


def amg_train_params_default():
    p = amg_train_params()
    load().amg_train_params_default(ctypes.byref(p))
    return p


def amg_learned_train(h, nn, params=None, stream=None):
    """Generate (residual, error) pairs with the solver and train nn on them; returns the batch losses."""
    p = params or amg_train_params_default()
    losses = np.zeros(max(1, p.npairs // p.batch), dtype=np.float64)
    _check(load().amg_learned_train(h, nn, ctypes.byref(p), losses.ctypes.data_as(_dp), _stream(stream)))
    return losses

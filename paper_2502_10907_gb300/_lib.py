"""ctypes binding of libmtf (include/mtf.h): argument marshalling only.

Every function here has the name and argument order of its C entry point;
host arrays are numpy arrays, device buffers are passed as integer device
pointers (e.g. ``tensor.data_ptr()``) and streams as integer handles.  A
non-OK status raises :class:`MtfError`.  The CUDA library must have been
built (``paper_2502_10907_gb300.build.build()``); there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB as _LIB_PATH

MTF_OK, MTF_ERR_ARG, MTF_ERR_MESH, MTF_ERR_CUDA, MTF_ERR_OOM, MTF_ERR_NOCONV, MTF_ERR_NAN, MTF_ERR_TIMEOUT = range(8)
MTF_PREC_FP64, MTF_PREC_MIXED = 0, 1
MTF_PRECOND_NONE, MTF_PRECOND_OSRC = 0, 1


class MtfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"libmtf status {status}: {msg}")
        self.status = status


class mtf_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("n_ss", ctypes.c_int32), ("restart", ctypes.c_int32),
                ("max_iter", ctypes.c_int32), ("tol", ctypes.c_double), ("precond", ctypes.c_int32),
                ("osrc_np", ctypes.c_int32), ("osrc_theta", ctypes.c_double),
                ("osrc_eps_scale", ctypes.c_double), ("max_refine", ctypes.c_int32), ("learned", ctypes.c_int32),
                ("osrc_half", ctypes.c_int32), ("recycle", ctypes.c_int32), ("residual_df", ctypes.c_int32),
                ("block_krylov", ctypes.c_int32), ("mv_tensor", ctypes.c_int32),
                ("residual_fp64", ctypes.c_int32), ("inner_tol_min", ctypes.c_double),
                ("gs_dots_half", ctypes.c_int32), ("osrc_type", ctypes.c_int32)]


class mtf_solve_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("restarts", ctypes.c_int32), ("refinements", ctypes.c_int32),
                ("converged", ctypes.c_int32), ("rel_residual", ctypes.c_double), ("seconds", ctypes.c_double),
                ("launch_seconds", ctypes.c_double), ("lsq_seconds", ctypes.c_double),
                ("wait_seconds", ctypes.c_double)]


_lib = None
_vp, _i32, _i64, _dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
_SIGS = {
    "mtf_nearfield": (_i32, [_vp, _vp, _i32, _vp, _vp, _i32, _vp, _vp]),
    "mtf_default_options": (None, [ctypes.POINTER(mtf_options)]),
    "mtf_mesh_create": (_i32, [_vp, _i32, _vp, _i32, _vp, _i32, ctypes.POINTER(_vp)]),
    "mtf_mesh_info": (_i32, [_vp, _vp, ctypes.POINTER(_i64)]),
    "mtf_mesh_pair_counts": (_i32, [_vp, _vp]),
    "mtf_mesh_destroy": (None, [_vp]),
    "mtf_assemble": (_i32, [_vp, _dbl, _vp, _vp, ctypes.POINTER(mtf_options), _vp, ctypes.POINTER(_vp)]),
    "mtf_reassemble": (_i32, [_vp, _dbl, _vp, _vp, _vp]),
    "mtf_profile_enable": (_i32, [_i32]),
    "mtf_profile_read": (_i32, [_i32, _vp, _vp]),
    "mtf_profile_read_bytes": (_i32, [_i32, _vp, _vp, _vp]),
    "mtf_kernel_count": (_i32, []),
    "mtf_kernel_name": (ctypes.c_char_p, [_i32]),
    "mtf_get_block": (_i32, [_vp, _i32, _vp, _vp, _vp]),
    "mtf_matvec": (_i32, [_vp, _vp, _vp, _i32, _vp]),
    "mtf_precond_apply": (_i32, [_vp, _vp, _vp, _i32, _vp]),
    "mtf_matvec_f32": (_i32, [_vp, _vp, _vp, _i32, _vp]),
    "mtf_matvec_adjoint_f32": (_i32, [_vp, _vp, _vp, _i32, _vp]),
    "mtf_precond_apply_f32": (_i32, [_vp, _vp, _vp, _i32, _vp]),
    "mtf_rhs": (_i32, [_vp, _i32, _vp, _vp, _vp, _vp]),
    "mtf_solve": (_i32, [_vp, _i32, _vp, _vp, _vp, ctypes.POINTER(mtf_solve_stats), _vp]),
    "mtf_solve_static": (_i32, [_vp, _i32, _vp, _vp, _vp, ctypes.POINTER(mtf_solve_stats), _vp]),
    "mtf_solve_rhs": (_i32, [_vp, _i32, _vp, _vp, ctypes.POINTER(mtf_solve_stats), _vp]),
    "mtf_solve_batch": (_i32, [_i32, _vp, _vp, _vp, _vp, _vp, ctypes.POINTER(mtf_solve_stats), _i32, _vp]),
    "mtf_autotune": (_i32, [_vp, _i32, _i32, ctypes.c_char_p, _i32, _vp]),
    "mtf_probe_peaks": (_i32, [_vp, _vp]),
    "mtf_farfield": (_i32, [_vp, _vp, _i32, _vp, _i32, _vp, _vp]),
    "mtf_system_destroy": (None, [_vp]),
    "mtf_learned_param_count": (_i64, [_vp]),
    "mtf_learned_init": (_i32, [_vp, _i32, ctypes.c_uint64]),
    "mtf_learned_get_params": (_i32, [_vp, _vp]),
    "mtf_learned_set_params": (_i32, [_vp, _vp]),
    "mtf_learned_features": (_i32, [_vp, _vp, _vp]),
    "mtf_learned_loss_grad": (_i32, [_vp, _vp, _vp, _vp, _i64, _vp, ctypes.POINTER(_dbl), _vp]),
    "mtf_learned_power_grad": (_i32, [_vp, _vp, _i32, _dbl, _dbl, _i32, _vp, ctypes.POINTER(_dbl), _vp]),
    "mtf_learned_stencil_adjoint": (_i32, [_vp, _vp, _vp, _vp, _i32, _vp]),
    "mtf_precond_adjoint_f32": (_i32, [_vp, _vp, _vp, _i32, _vp]),
    "mtf_learned_centre": (_dbl, [_vp, ctypes.POINTER(_dbl)]),
    "mtf_learned_train": (_i32, [_vp, _i32, _dbl, _i32, _i32, ctypes.c_uint64, ctypes.POINTER(_dbl),
                                 ctypes.POINTER(_dbl), _vp]),
    "mtf_learned_fit": (_i32, [_vp, _i32, _vp, _vp, _i32, _i32, _dbl, _i32, _i32, ctypes.c_uint64, _vp, _vp]),
    "mtf_learned_enable": (_i32, [_vp, _i32]),
    "mtf_learned_apply": (_i32, [_vp, _vp, _vp, _i32, _vp]),
    "mtf_status_string": (ctypes.c_char_p, [_i32]),
    "mtf_last_error": (ctypes.c_char_p, []),
}


def lib_path() -> str:
    return _LIB_PATH


def load():
    """Load libmtf.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"{_LIB_PATH} is missing: build the CUDA library first "
                               "(python -c 'import __graft_entry__ as g; g.build()')")
        lib = ctypes.CDLL(_LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def exported_symbols():
    return list(_SIGS)


def _check(st):
    if st != MTF_OK:
        raise MtfError(st, load().mtf_last_error().decode())


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, int):
        return a
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    raise TypeError(type(a))


def mtf_default_options() -> mtf_options:
    o = mtf_options()
    load().mtf_default_options(ctypes.byref(o))
    return o


def mtf_mesh_create(vertices, triangles, labels, n_domains):
    V = np.ascontiguousarray(vertices, dtype=np.float64)
    F = np.ascontiguousarray(triangles, dtype=np.int32)
    L = np.ascontiguousarray(labels, dtype=np.int32)
    h = _vp()
    _check(load().mtf_mesh_create(_ptr(V), len(V), _ptr(F), len(F), _ptr(L), int(n_domains), ctypes.byref(h)))
    return h.value


def mtf_mesh_info(mesh, n_domains):
    nd = np.zeros(n_domains, dtype=np.int32)
    nt = _i64()
    _check(load().mtf_mesh_info(mesh, _ptr(nd), ctypes.byref(nt)))
    return nd, int(nt.value)


def mtf_mesh_pair_counts(mesh):
    c = np.zeros(4, dtype=np.int64)
    _check(load().mtf_mesh_pair_counts(mesh, _ptr(c)))
    return c


def mtf_mesh_destroy(mesh):
    load().mtf_mesh_destroy(mesh)


def mtf_assemble(mesh, k0, eps_r, mu_r, opt=None, stream=0):
    e = np.ascontiguousarray(eps_r, dtype=np.float64)
    m = np.ascontiguousarray(mu_r, dtype=np.float64)
    h = _vp()
    _check(load().mtf_assemble(mesh, float(k0), _ptr(e), _ptr(m), ctypes.byref(opt) if opt is not None else None,
                               stream or None, ctypes.byref(h)))
    return h.value


def mtf_reassemble(sys_, k0, eps_r, mu_r, stream=0):
    e = np.ascontiguousarray(eps_r, dtype=np.float64)
    m = np.ascontiguousarray(mu_r, dtype=np.float64)
    _check(load().mtf_reassemble(sys_, float(k0), _ptr(e), _ptr(m), stream or None))


def mtf_profile_enable(on):
    _check(load().mtf_profile_enable(1 if on else 0))


def mtf_kernel_count():
    return int(load().mtf_kernel_count())


def mtf_kernel_name(i):
    return load().mtf_kernel_name(int(i)).decode()


def mtf_profile_read():
    """Returns {kernel name: (launches, ms)} since the last read, and resets."""
    n = mtf_kernel_count()
    la = np.zeros(n, dtype=np.int64)
    ms = np.zeros(n, dtype=np.float64)
    _check(load().mtf_profile_read(n, _ptr(la), _ptr(ms)))
    return {mtf_kernel_name(i): (int(la[i]), float(ms[i])) for i in range(n)}


def mtf_profile_read_bytes():
    """Returns {kernel name: (launches, ms, algorithmic bytes)} since the last read, and resets."""
    n = mtf_kernel_count()
    la = np.zeros(n, dtype=np.int64)
    ms = np.zeros(n, dtype=np.float64)
    by = np.zeros(n, dtype=np.float64)
    _check(load().mtf_profile_read_bytes(n, _ptr(la), _ptr(ms), _ptr(by)))
    return {mtf_kernel_name(i): (int(la[i]), float(ms[i]), float(by[i])) for i in range(n)}


def mtf_get_block(sys_, i, t_out, k_out, stream=0):
    _check(load().mtf_get_block(sys_, int(i), _ptr(t_out), _ptr(k_out), stream or None))


def mtf_matvec(sys_, x, y, nrhs, stream=0):
    _check(load().mtf_matvec(sys_, _ptr(x), _ptr(y), int(nrhs), stream or None))


def mtf_precond_apply(sys_, r, z, nrhs, stream=0):
    _check(load().mtf_precond_apply(sys_, _ptr(r), _ptr(z), int(nrhs), stream or None))


def mtf_matvec_f32(sys_, x, y, nrhs, stream=0):
    _check(load().mtf_matvec_f32(sys_, _ptr(x), _ptr(y), int(nrhs), stream or None))


def mtf_matvec_adjoint_f32(sys_, v, y, nrhs, stream=0):
    _check(load().mtf_matvec_adjoint_f32(sys_, _ptr(v), _ptr(y), int(nrhs), stream or None))


def mtf_precond_apply_f32(sys_, r, z, nrhs, stream=0):
    _check(load().mtf_precond_apply_f32(sys_, _ptr(r), _ptr(z), int(nrhs), stream or None))


def mtf_rhs(sys_, dirs, pols, b_out, stream=0):
    d = np.ascontiguousarray(dirs, dtype=np.float64)
    p = np.ascontiguousarray(pols, dtype=np.complex128)
    _check(load().mtf_rhs(sys_, len(d), _ptr(d), _ptr(p), _ptr(b_out), stream or None))


def mtf_solve(sys_, dirs, pols, x_out, stream=0, raise_on_noconv=True):
    d = np.ascontiguousarray(dirs, dtype=np.float64)
    p = np.ascontiguousarray(pols, dtype=np.complex128)
    st = mtf_solve_stats()
    status = load().mtf_solve(sys_, len(d), _ptr(d), _ptr(p), _ptr(x_out), ctypes.byref(st), stream or None)
    if status != MTF_OK and (raise_on_noconv or status != MTF_ERR_NOCONV):
        _check(status)
    return st, status


def mtf_solve_rhs(sys_, b, x_out, stream=0, raise_on_noconv=True):
    """Solve M x = b for device right-hand sides b (nrhs, n_total) complex128."""
    st = mtf_solve_stats()
    status = load().mtf_solve_rhs(sys_, int(b.shape[0]), _ptr(b), _ptr(x_out), ctypes.byref(st), stream or None)
    if status != MTF_OK and (raise_on_noconv or status != MTF_ERR_NOCONV):
        _check(status)
    return st, status


def mtf_solve_batch(systems, dirs_list, pols_list, x_outs, threads=0, stream=0, raise_on_noconv=True):
    """Instances solved concurrently: systems[i] with waves dirs_list[i], pols_list[i] into x_outs[i]."""
    n = len(systems)
    ds = [np.ascontiguousarray(d, dtype=np.float64) for d in dirs_list]
    ps = [np.ascontiguousarray(p, dtype=np.complex128) for p in pols_list]
    sysv = (ctypes.c_void_p * n)(*systems)
    nr = (ctypes.c_int32 * n)(*[len(d) for d in ds])
    dv = (ctypes.c_void_p * n)(*[_ptr(d) for d in ds])
    pv = (ctypes.c_void_p * n)(*[_ptr(p) for p in ps])
    xv = (ctypes.c_void_p * n)(*[_ptr(x) for x in x_outs])
    st = (mtf_solve_stats * n)()
    status = load().mtf_solve_batch(n, sysv, nr, dv, pv, xv, st, int(threads), stream or None)
    if status != MTF_OK and (raise_on_noconv or status != MTF_ERR_NOCONV):
        _check(status)
    return list(st), status


def mtf_probe_peaks(stream=0):
    """Measured (FP32 FLOP/s, FP64 FLOP/s, SFU results/s) of the current device."""
    r = np.zeros(3, dtype=np.float64)
    _check(load().mtf_probe_peaks(_ptr(r), stream or None))
    return tuple(float(v) for v in r)


def mtf_autotune(sys_, nrhs, reps=5, stream=0):
    """Times the apply plans for nrhs right-hand sides, keeps the fastest; returns the report lines."""
    buf = ctypes.create_string_buffer(4096)
    _check(load().mtf_autotune(sys_, int(nrhs), int(reps), buf, len(buf), stream or None))
    return buf.value.decode().strip().split("\n")


def mtf_solve_static(sys_, dirs, pols, x_out, stream=0, raise_on_noconv=True):
    """mtf_solve that allocates no device memory (static 16 MiB workspace)."""
    d = np.ascontiguousarray(dirs, dtype=np.float64)
    p = np.ascontiguousarray(pols, dtype=np.complex128)
    st = mtf_solve_stats()
    status = load().mtf_solve_static(sys_, len(d), _ptr(d), _ptr(p), _ptr(x_out), ctypes.byref(st),
                                     stream or None)
    if status != MTF_OK and (raise_on_noconv or status != MTF_ERR_NOCONV):
        _check(status)
    return st, status


def mtf_farfield(sys_, x, nrhs, obs_dirs, f_out, stream=0):
    o = np.ascontiguousarray(obs_dirs, dtype=np.float64)
    _check(load().mtf_farfield(sys_, _ptr(x), int(nrhs), _ptr(o), len(o), _ptr(f_out), stream or None))


def mtf_nearfield(sys_, x, nrhs, points, domains, f_out, stream=0):
    pts = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 3)
    dom = np.ascontiguousarray(domains, dtype=np.int32).reshape(-1)
    if len(dom) != len(pts):
        raise ValueError("one subdomain per point")
    _check(load().mtf_nearfield(sys_, _ptr(x), int(nrhs), _ptr(pts), _ptr(dom), len(pts), _ptr(f_out),
                                stream or None))


def mtf_system_destroy(sys_):
    load().mtf_system_destroy(sys_)


# --- learned correction of block-OSRC ---------------------------------------
LEARNED_KINDS = {"table": 0, "network": 1}


class mtf_learned_report(ctypes.Structure):
    _fields_ = [("plain_iterations", ctypes.c_int32), ("best_iterations", ctypes.c_int32),
                ("best_round", ctypes.c_int32), ("rounds", ctypes.c_int32), ("loss_first", ctypes.c_double),
                ("loss_last", ctypes.c_double), ("enabled", ctypes.c_int32)]


def mtf_learned_param_count(sys_):
    return int(load().mtf_learned_param_count(sys_))


def mtf_learned_init(sys_, kind="table", seed=0):
    _check(load().mtf_learned_init(sys_, LEARNED_KINDS[kind], int(seed)))


def mtf_learned_get_params(sys_):
    out = np.zeros(mtf_learned_param_count(sys_), dtype=np.float32)
    _check(load().mtf_learned_get_params(sys_, _ptr(out)))
    return out


def mtf_learned_set_params(sys_, params):
    p = np.ascontiguousarray(params, dtype=np.float32)
    if p.size != mtf_learned_param_count(sys_):
        raise ValueError("wrong number of parameters")
    _check(load().mtf_learned_set_params(sys_, _ptr(p)))


def mtf_learned_features(sys_, x_out, stream=0):
    _check(load().mtf_learned_features(sys_, _ptr(x_out), stream or None))


def mtf_learned_loss_grad(sys_, x, t, w, rows, grad_out, stream=0):
    loss = _dbl()
    _check(load().mtf_learned_loss_grad(sys_, _ptr(x), _ptr(t), _ptr(w), int(rows), _ptr(grad_out),
                                        ctypes.byref(loss), stream or None))
    return loss.value


def mtf_learned_power_grad(sys_, z, ncols, c0, K, grad_out, stream=0):
    loss = _dbl()
    _check(load().mtf_learned_power_grad(sys_, _ptr(z), int(ncols), float(np.real(c0)), float(np.imag(c0)), int(K),
                                         _ptr(grad_out), ctypes.byref(loss), stream or None))
    return loss.value


def mtf_learned_stencil_adjoint(sys_, w, out_r, out_p, nrhs, stream=0):
    _check(load().mtf_learned_stencil_adjoint(sys_, _ptr(w), _ptr(out_r), _ptr(out_p), int(nrhs), stream or None))


def mtf_precond_adjoint_f32(sys_, w, z, nrhs, stream=0):
    _check(load().mtf_precond_adjoint_f32(sys_, _ptr(w), _ptr(z), int(nrhs), stream or None))


def mtf_learned_centre(sys_):
    im = _dbl()
    re = load().mtf_learned_centre(sys_, ctypes.byref(im))
    return complex(re, im.value)


def mtf_learned_train(sys_, steps, lr, batch, K, seed=0, stream=0):
    a, b = _dbl(), _dbl()
    _check(load().mtf_learned_train(sys_, int(steps), float(lr), int(batch), int(K), int(seed), ctypes.byref(a),
                                    ctypes.byref(b), stream or None))
    return a.value, b.value


def mtf_learned_fit(sys_, dirs, pols, rounds, steps_per_round, lr, batch, K, seed=0, stream=0):
    d = np.ascontiguousarray(dirs, dtype=np.float64).reshape(-1, 3)
    p = np.ascontiguousarray(pols, dtype=np.complex128).reshape(len(d), 3)
    rep = mtf_learned_report()
    _check(load().mtf_learned_fit(sys_, len(d), _ptr(d), _ptr(p), int(rounds), int(steps_per_round), float(lr),
                                  int(batch), int(K), int(seed), ctypes.byref(rep), stream or None))
    return {f: getattr(rep, f) for f, _ in mtf_learned_report._fields_}


def mtf_learned_enable(sys_, on):
    _check(load().mtf_learned_enable(sys_, 1 if on else 0))


def mtf_learned_apply(sys_, r, z, nrhs, stream=0):
    _check(load().mtf_learned_apply(sys_, _ptr(r), _ptr(z), int(nrhs), stream or None))

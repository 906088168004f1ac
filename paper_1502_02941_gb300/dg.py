"""ctypes binding of libdg (include/dg.h): argument marshalling only.

Every entry point of the C ABI is exposed under its own name with the same
arguments; device pointers may be passed as torch tensors (their data_ptr() is
used) or as integers, host arrays as numpy arrays.  ``DG`` is a thin object
wrapper that owns one handle and issues work on torch's current stream.

There is no fallback: if libdg.so has not been built, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libdg.so")
HEADER = os.path.join(os.path.dirname(_PKG), "include", "dg.h")

# constants mirrored from include/dg.h
DG_OK, DG_ERR_INVALID_ARG, DG_ERR_CUDA, DG_NOT_CONVERGED = 0, 1, 2, 3
DG_ERR_TIMEOUT, DG_ERR_NONFINITE, DG_ERR_SINGULAR_BLOCK, DG_ERR_MESH = 4, 5, 6, 7
DG_ERR_STATE, DG_ERR_NOMEM = 8, 9
DG_NIPG, DG_SIPG, DG_IIPG = 1, 2, 3
DG_F64, DG_F32, DG_BF16 = 0, 1, 2
DG_STORE_F64, DG_STORE_F32, DG_STORE_BF16 = 1, 2, 4
DG_PRECOND_NONE, DG_PRECOND_BLOCK_JACOBI, DG_PRECOND_MLP, DG_PRECOND_SCHWARZ = 0, 1, 2, 3
DG_POINTS_VOLUME, DG_POINTS_BOUNDARY, DG_POINTS_ERROR, DG_POINTS_FACE = 0, 1, 2, 3
DG_PROF_DOTS, DG_PROF_UPDATE, DG_PROF_APPLY = 1, 2, 3
DG_WS_TOTAL, DG_WS_MESH, DG_WS_OPERATOR, DG_WS_PRECOND, DG_WS_SOLVER, DG_WS_LEARNED, DG_WS_SCRATCH, DG_WS_PEAK = range(8)

c_int32, c_int64, c_double, c_void_p = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p


class dg_params(ctypes.Structure):
    _fields_ = [("method", c_int32), ("degree", c_int32), ("sigma_int", c_double),
                ("sigma_bdry_factor", c_double), ("b0", c_double), ("store", c_int32),
                ("gmres_m", c_int32), ("tol", c_double), ("max_it", c_int32), ("precond", c_int32)]


class dg_coeffs(ctypes.Structure):
    _fields_ = [("eps", c_double), ("alpha", c_double), ("b", c_double * 6),
                ("f", c_void_p), ("f_const", c_double),
                ("gD", c_void_p), ("gD_const", c_double),
                ("gN", c_void_p), ("gN_const", c_double),
                ("eps_q", c_void_p), ("eps_f", c_void_p)]


class dg_info(ctypes.Structure):
    _fields_ = [("ne", c_int32), ("nv", c_int32), ("n_bedges", c_int32), ("n_interior", c_int32),
                ("nb", c_int32), ("dofs", c_int64), ("q_volume", c_int32), ("q_edge", c_int32),
                ("q_error", c_int32), ("block_bytes", c_int64 * 3)]


class dg_solve_info(ctypes.Structure):
    _fields_ = [("iterations", c_int32), ("restarts", c_int32), ("outer", c_int32),
                ("status", c_int32), ("relres", c_double)]


# dg_alloc_fn / dg_free_fn of include/dg.h
DG_ALLOC_FN = ctypes.CFUNCTYPE(c_void_p, c_void_p, ctypes.c_size_t, ctypes.c_int, c_void_p)
DG_FREE_FN = ctypes.CFUNCTYPE(None, c_void_p, c_void_p, ctypes.c_size_t, ctypes.c_int, c_void_p)

_lib = None

_SIGS = {
    "dg_set_allocator": (ctypes.c_int, [c_void_p, DG_ALLOC_FN, DG_FREE_FN, c_void_p]),
    "dg_set_arena": (ctypes.c_int, [c_void_p, c_void_p, ctypes.c_size_t]),
    "dg_workspace_size": (ctypes.c_size_t, [c_void_p, ctypes.c_int]),
    "dg_create": (ctypes.c_int, [ctypes.POINTER(c_void_p), ctypes.c_int, c_void_p]),
    "dg_destroy": (ctypes.c_int, [c_void_p]),
    "dg_set_stream": (ctypes.c_int, [c_void_p, c_void_p]),
    "dg_stream_create": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(c_void_p)]),
    "dg_stream_destroy": (ctypes.c_int, [c_void_p]),
    "dg_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "dg_last_error": (ctypes.c_char_p, [c_void_p]),
    "dg_params_default": (ctypes.c_int, [ctypes.POINTER(dg_params)]),
    "dg_mesh_upload": (ctypes.c_int, [c_void_p, c_void_p, ctypes.c_int, c_void_p, ctypes.c_int,
                                      c_void_p, ctypes.c_int, c_void_p, ctypes.c_int]),
    "dg_set_params": (ctypes.c_int, [c_void_p, ctypes.POINTER(dg_params)]),
    "dg_get_info": (ctypes.c_int, [c_void_p, ctypes.POINTER(dg_info)]),
    "dg_quad_points": (ctypes.c_int, [c_void_p, ctypes.c_int, c_void_p]),
    "dg_boundary_info": (ctypes.c_int, [c_void_p, c_void_p, c_void_p]),
    "dg_assemble": (ctypes.c_int, [c_void_p, ctypes.POINTER(dg_coeffs)]),
    "dg_get_rhs": (ctypes.c_int, [c_void_p, c_void_p]),
    "dg_get_blocks": (ctypes.c_int, [c_void_p, ctypes.c_int, c_void_p, c_void_p]),
    "dg_apply": (ctypes.c_int, [c_void_p, ctypes.c_int, c_void_p, c_void_p]),
    "dg_precond_setup": (ctypes.c_int, [c_void_p, ctypes.c_int]),
    "dg_precond_apply": (ctypes.c_int, [c_void_p, ctypes.c_int, c_void_p, c_void_p]),
    "dg_gmres_solve": (ctypes.c_int, [c_void_p, c_void_p, c_void_p, ctypes.POINTER(dg_solve_info)]),
    "dg_dense_solve": (ctypes.c_int, [c_void_p, c_void_p, c_void_p]),
    "dg_mixed_solve": (ctypes.c_int, [c_void_p, ctypes.c_int, ctypes.c_int, c_double, ctypes.c_int, c_void_p,
                                      c_void_p, ctypes.POINTER(dg_solve_info)]),
    "dg_gmres_ir_solve": (ctypes.c_int, [c_void_p, ctypes.c_int, ctypes.c_int, c_double, ctypes.c_int, c_void_p,
                                         c_void_p, ctypes.POINTER(dg_solve_info)]),
    "dg_l2_error": (ctypes.c_int, [c_void_p, c_void_p, c_void_p, ctypes.POINTER(c_double),
                                   ctypes.POINTER(c_double)]),
    "dg_eval": (ctypes.c_int, [c_void_p, c_void_p, ctypes.c_int, c_void_p, c_void_p]),
    "dg_l2_error_noalloc": (ctypes.c_int, [c_void_p, c_void_p, c_void_p, ctypes.POINTER(c_double),
                                           ctypes.POINTER(c_double)]),
    "dg_profile_kernel": (ctypes.c_int, [c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.POINTER(c_double)]),
    "dg_batch_setup": (ctypes.c_int, [c_void_p, ctypes.c_int, c_void_p, c_void_p]),
    "dg_batch_clear": (ctypes.c_int, [c_void_p]),
    "dg_batch_autotune": (ctypes.c_int, [c_void_p, ctypes.POINTER(ctypes.c_int)]),
    "dg_batch_set_tile": (ctypes.c_int, [c_void_p, ctypes.c_int]),
    "dg_batch_solve": (ctypes.c_int, [c_void_p, ctypes.c_int, ctypes.c_int, c_double, ctypes.c_int, c_void_p,
                                      c_void_p, c_void_p, c_void_p, c_void_p]),
    "dg_batch_gmres_ir_solve": (ctypes.c_int, [c_void_p, ctypes.c_int, ctypes.c_int, c_double, ctypes.c_int,
                                               c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "dg_batch_group_solve": (ctypes.c_int, [c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, c_double,
                                            ctypes.c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "dg_batch_group_gmres_ir_solve": (ctypes.c_int, [c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, c_double,
                                                     ctypes.c_int, c_void_p, c_void_p, c_void_p, c_void_p,
                                                     c_void_p]),
    "dg_mesh_refine": (ctypes.c_int, [c_void_p, ctypes.c_int, c_void_p, ctypes.c_int, c_void_p, ctypes.c_int,
                                      c_void_p, ctypes.c_int, c_void_p, ctypes.POINTER(ctypes.c_int), c_void_p,
                                      ctypes.POINTER(ctypes.c_int), c_void_p, ctypes.POINTER(ctypes.c_int),
                                      c_void_p, ctypes.POINTER(ctypes.c_int)]),
    "dg_nonlinear_global": (ctypes.c_int, [c_void_p, ctypes.c_int, c_double, c_void_p, c_void_p, c_void_p]),
    "dg_newton_solve": (ctypes.c_int, [c_void_p, ctypes.c_int, c_double, ctypes.c_int, c_double, c_void_p,
                                       c_void_p, ctypes.POINTER(dg_solve_info)]),
    "dg_mlp_num_params": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(c_int64)]),
    "dg_mlp_init": (ctypes.c_int, [c_void_p, ctypes.c_uint64]),
    "dg_mlp_set_weights": (ctypes.c_int, [c_void_p, c_void_p, c_int64]),
    "dg_mlp_get_weights": (ctypes.c_int, [c_void_p, c_void_p, c_int64]),
    "dg_mlp_collect": (ctypes.c_int, [c_void_p, c_void_p, c_void_p]),
    "dg_mlp_collect_basis": (ctypes.c_int, [c_void_p, ctypes.c_int]),
    "dg_mlp_num_rows": (ctypes.c_int, [c_void_p, ctypes.POINTER(c_int64)]),
    "dg_mlp_get_rows": (ctypes.c_int, [c_void_p, c_void_p, c_void_p, c_int64]),
    "dg_mlp_clear_data": (ctypes.c_int, [c_void_p]),
    "dg_mlp_train": (ctypes.c_int, [c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_float, ctypes.c_uint64, c_void_p]),
    "dg_mlp_loss_grad": (ctypes.c_int, [c_void_p, c_void_p, c_void_p, ctypes.c_int, ctypes.POINTER(c_double),
                                        c_void_p]),
    "dg_mlp_forward": (ctypes.c_int, [c_void_p, c_void_p, ctypes.c_int, c_void_p]),
    "dg_get_launch_count": (ctypes.c_int, [c_void_p, ctypes.POINTER(c_int64)]),
    "dg_reference_basis": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, c_void_p, c_void_p, c_void_p, c_void_p]),
    "dg_reference_rule": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, c_void_p, c_void_p,
                                         ctypes.POINTER(ctypes.c_int)]),
}


def header_symbols():
    """Entry points declared in include/dg.h."""
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:dg_status|const char\*|size_t)\s+(dg_\w+)\s*\(", txt, re.M)))


def load():
    """Load libdg.so; raises if it is missing (no fallback path exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is not built: run `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class DGError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{status_name(status)}: {msg}")
        self.status = status


def status_name(s):
    return load().dg_status_string(int(s)).decode()


_TORCH_DTYPES = {"f64": "torch.float64", "f32": "torch.float32", "bf16": "torch.bfloat16", "i32": "torch.int32"}
_NP_DTYPES = {"f64": np.float64, "f32": np.float32, "i32": np.int32}


def _host(x, n=None, dtype=None, what="host argument"):
    """Pointer of HOST data: a C-contiguous numpy array (or a contiguous CPU
    torch tensor), an integer address (passed through unchecked) or None.  A
    CUDA tensor is refused: the library reads or writes this memory from the
    CPU.  n: least number of elements; dtype: "f64" / "f32" / "i32"."""
    if x is None or isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError(f"{what}: array must be C-contiguous")
        if dtype is not None and x.dtype != _NP_DTYPES[dtype]:
            raise ValueError(f"{what}: numpy dtype {_NP_DTYPES[dtype].__name__} expected, got {x.dtype}")
        if n is not None and x.size < n:
            raise ValueError(f"{what}: {n} elements needed, the array has {x.size}")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if x.is_cuda:
            raise ValueError(f"{what}: host memory is expected here (a numpy array), not a CUDA tensor")
        if not x.is_contiguous():
            raise ValueError(f"{what}: tensor must be contiguous")
        if dtype is not None and str(x.dtype) != _TORCH_DTYPES[dtype]:
            raise ValueError(f"{what}: {_TORCH_DTYPES[dtype]} expected, got {x.dtype}")
        if n is not None and x.numel() < n:
            raise ValueError(f"{what}: {n} elements needed, the tensor has {x.numel()}")
        return x.data_ptr()
    raise TypeError(f"{what}: cannot take a pointer of {type(x)}")


def _dev(x, n=None, dtype=None, what="device argument"):
    """Pointer of DEVICE data: a contiguous CUDA torch tensor, an integer
    address (a raw device pointer, passed through unchecked) or None.  numpy
    arrays and CPU tensors are refused here, because the kernels would
    dereference their host addresses.  n: least number of elements; dtype:
    "f64" / "f32" / "bf16" / "i32" (a tuple allows several)."""
    if x is None or isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        raise ValueError(f"{what}: device memory is expected here (a CUDA tensor), not a numpy array")
    if hasattr(x, "data_ptr"):
        if not x.is_cuda:
            raise ValueError(f"{what}: a device (CUDA) tensor is expected here; host data goes in numpy arrays")
        if not x.is_contiguous():
            raise ValueError(f"{what}: tensor must be contiguous")
        if dtype is not None:
            allowed = (dtype,) if isinstance(dtype, str) else dtype
            if str(x.dtype) not in [_TORCH_DTYPES[d] for d in allowed]:
                raise ValueError(f"{what}: {' or '.join(_TORCH_DTYPES[d] for d in allowed)} expected, got {x.dtype}")
        if n is not None and x.numel() < n:
            raise ValueError(f"{what}: {n} elements needed, the tensor has {x.numel()}")
        return x.data_ptr()
    raise TypeError(f"{what}: cannot take a pointer of {type(x)}")


def _sizes(h):
    """Mesh sizes of handle h under its current parameters, or None when the
    library has none yet (it then reports the call-order error itself)."""
    i = dg_info()
    if load().dg_get_info(h, ctypes.byref(i)) != DG_OK:
        return None
    return i


def _vec_dtype(dtype):
    return "f64" if int(dtype) == DG_F64 else "f32"


# ---------------------------------------------------------------------------
# the C ABI under its own names
# ---------------------------------------------------------------------------
def dg_create(device=0, stream=None):
    h = c_void_p()
    s = load().dg_create(ctypes.byref(h), int(device), stream)
    if s != DG_OK:
        raise DGError(s, "dg_create failed")
    return h


def dg_destroy(h):
    return load().dg_destroy(h)


def dg_set_stream(h, stream):
    return load().dg_set_stream(h, stream)


def dg_stream_create(device=0):
    st = c_void_p()
    s = load().dg_stream_create(int(device), ctypes.byref(st))
    if s != DG_OK:
        raise DGError(s, "dg_stream_create failed")
    return st.value


def dg_stream_destroy(stream):
    return load().dg_stream_destroy(stream)


def dg_status_string(s):
    return load().dg_status_string(int(s)).decode()


def dg_last_error(h):
    return load().dg_last_error(h).decode()


def dg_params_default():
    p = dg_params()
    load().dg_params_default(ctypes.byref(p))
    return p


def dg_mesh_upload(h, nodes, elems, dirichlet, neumann):
    nodes = np.ascontiguousarray(nodes, dtype=np.float64).reshape(-1, 2)
    elems = np.ascontiguousarray(elems, dtype=np.int32).reshape(-1, 3)
    dirichlet = np.ascontiguousarray(dirichlet, dtype=np.int32).reshape(-1, 2)
    neumann = np.ascontiguousarray(neumann, dtype=np.int32).reshape(-1, 2)
    return load().dg_mesh_upload(h, _host(nodes), nodes.shape[0], _host(elems), elems.shape[0],
                                 _host(dirichlet) if len(dirichlet) else None, dirichlet.shape[0],
                                 _host(neumann) if len(neumann) else None, neumann.shape[0])


def dg_set_params(h, p):
    return load().dg_set_params(h, ctypes.byref(p))


def dg_set_allocator(h, alloc_fn, free_fn, ctx=None):
    """alloc_fn / free_fn: DG_ALLOC_FN / DG_FREE_FN objects (the caller keeps
    them alive as long as the handle), or None for both (cudaMalloc)."""
    return load().dg_set_allocator(h, alloc_fn if alloc_fn is not None else DG_ALLOC_FN(),
                                   free_fn if free_fn is not None else DG_FREE_FN(), ctx)


def dg_set_arena(h, base, nbytes):
    return load().dg_set_arena(h, _dev(base, None, None, "arena"), int(nbytes))


def dg_workspace_size(h, what):
    return int(load().dg_workspace_size(h, int(what)))


def dg_get_info(h):
    i = dg_info()
    s = load().dg_get_info(h, ctypes.byref(i))
    return s, i


def _points_count(i, which):
    return {DG_POINTS_VOLUME: i.ne * i.q_volume, DG_POINTS_BOUNDARY: i.n_bedges * i.q_edge,
            DG_POINTS_ERROR: i.ne * i.q_error, DG_POINTS_FACE: i.ne * 3 * i.q_edge}.get(int(which))


def dg_quad_points(h, which, xy):
    i = _sizes(h)
    n = None if i is None or _points_count(i, which) is None else 2 * _points_count(i, which)
    return load().dg_quad_points(h, int(which), _dev(xy, n, "f64", "xy"))


def dg_boundary_info(h, normals, types=None):
    i = _sizes(h)
    nbe = None if i is None else i.n_bedges
    return load().dg_boundary_info(h, _dev(normals, None if nbe is None else 2 * nbe, "f64", "normals"),
                                   _dev(types, nbe, "i32", "type"))


def dg_coeffs_data(h, c, f=None, gD=None, gN=None, eps_q=None, eps_f=None):
    """Fill the device pointers of a dg_coeffs from tensors (checked against
    the handle's point counts)."""
    i = _sizes(h)
    nv = None if i is None else i.ne * i.q_volume
    ne_ = None if i is None else i.n_bedges * i.q_edge
    nf = None if i is None else i.ne * 3 * i.q_edge
    c.f, c.gD, c.gN = _dev(f, nv, "f64", "f"), _dev(gD, ne_, "f64", "gD"), _dev(gN, ne_, "f64", "gN")
    c.eps_q, c.eps_f = _dev(eps_q, nv, "f64", "eps_q"), _dev(eps_f, nf, "f64", "eps_f")
    return c


def dg_assemble(h, c):
    return load().dg_assemble(h, ctypes.byref(c))


def _dofs(h):
    i = _sizes(h)
    return None if i is None else i.dofs


def dg_get_rhs(h, F):
    return load().dg_get_rhs(h, _dev(F, _dofs(h), "f64", "F"))


def dg_get_blocks(h, dtype, out, nbr=None):
    i = _sizes(h)
    n = None if i is None else i.ne * 4 * i.nb * i.nb
    kinds = {DG_F64: "f64", DG_F32: "f32", DG_BF16: "bf16"}.get(int(dtype))
    return load().dg_get_blocks(h, int(dtype), _dev(out, n, kinds, "out"),
                                _dev(nbr, None if i is None else 3 * i.ne, "i32", "nbr"))


def dg_apply(h, dtype, x, y):
    n, t = _dofs(h), _vec_dtype(dtype)
    return load().dg_apply(h, int(dtype), _dev(x, n, t, "x"), _dev(y, n, t, "y"))


def dg_precond_setup(h, kind):
    return load().dg_precond_setup(h, int(kind))


def dg_precond_apply(h, dtype, r, z):
    n, t = _dofs(h), _vec_dtype(dtype)
    return load().dg_precond_apply(h, int(dtype), _dev(r, n, t, "r"), _dev(z, n, t, "z"))


def _solve_vectors(h, F, x):
    n = _dofs(h)
    return _dev(F, n, "f64", "F"), _dev(x, n, "f64", "x")


def dg_gmres_solve(h, F, x, info=None):
    Fp, xp = _solve_vectors(h, F, x)
    return load().dg_gmres_solve(h, Fp, xp, ctypes.byref(info) if info is not None else None)


def dg_mixed_solve(h, inner_dtype, inner_m, inner_tol, max_outer, F, x, info=None):
    Fp, xp = _solve_vectors(h, F, x)
    return load().dg_mixed_solve(h, int(inner_dtype), int(inner_m), float(inner_tol), int(max_outer), Fp, xp,
                                 ctypes.byref(info) if info is not None else None)


def dg_gmres_ir_solve(h, inner_dtype, inner_m, inner_tol, max_outer, F, x, info=None):
    Fp, xp = _solve_vectors(h, F, x)
    return load().dg_gmres_ir_solve(h, int(inner_dtype), int(inner_m), float(inner_tol), int(max_outer), Fp, xp,
                                    ctypes.byref(info) if info is not None else None)


def dg_dense_solve(h, F, x):
    Fp, xp = _solve_vectors(h, F, x)
    return load().dg_dense_solve(h, Fp, xp)


def _l2_args(h, x, uex_q):
    i = _sizes(h)
    return (_dev(x, None if i is None else i.dofs, "f64", "x"),
            _dev(uex_q, None if i is None else i.ne * i.q_error, "f64", "uex_q"))


def dg_l2_error(h, x, uex_q):
    l2, hmax = c_double(), c_double()
    s = load().dg_l2_error(h, *_l2_args(h, x, uex_q), ctypes.byref(l2), ctypes.byref(hmax))
    return s, l2.value, hmax.value


def dg_l2_error_noalloc(h, x, uex_q):
    """dg_l2_error through the allocation-free entry point (see include/dg.h)."""
    l2, hmax = c_double(), c_double()
    s = load().dg_l2_error_noalloc(h, *_l2_args(h, x, uex_q), ctypes.byref(l2), ctypes.byref(hmax))
    return s, l2.value, hmax.value


def dg_eval(h, x, rs, out):
    rs = np.ascontiguousarray(rs, dtype=np.float64).reshape(-1, 2)
    i = _sizes(h)
    return load().dg_eval(h, _dev(x, None if i is None else i.dofs, "f64", "x"), rs.shape[0], _host(rs),
                          _dev(out, None if i is None else i.ne * rs.shape[0], "f64", "out"))


def dg_profile_kernel(h, which, dtype, param, reps):
    ms = c_double()
    s = load().dg_profile_kernel(h, int(which), int(dtype), int(param), int(reps), ctypes.byref(ms))
    return s, ms.value


def dg_batch_setup(h, elem_start, coeffs):
    elem_start = np.ascontiguousarray(elem_start, dtype=np.int32).reshape(-1)
    coeffs = np.ascontiguousarray(coeffs, dtype=np.float64).reshape(-1, 8)
    if coeffs.shape[0] != elem_start.shape[0] - 1:
        raise ValueError("coeffs needs one row of 8 per instance")
    return load().dg_batch_setup(h, elem_start.shape[0] - 1, _host(elem_start), _host(coeffs))


def dg_batch_clear(h):
    return load().dg_batch_clear(h)


def dg_batch_autotune(h):
    t = ctypes.c_int()
    s = load().dg_batch_autotune(h, ctypes.byref(t))
    return s, t.value


def dg_batch_set_tile(h, tile):
    return load().dg_batch_set_tile(h, int(tile))


def _batch_outputs(its, relres, status, n_inst):
    return (_host(its, n_inst, "i32", "its"), _host(relres, n_inst, "f64", "relres"),
            _host(status, n_inst, "i32", "status"))


def dg_batch_solve(h, inner_dtype, inner_m, inner_tol, max_outer, F, x, its=None, relres=None, status=None,
                   n_inst=None):
    Fp, xp = _solve_vectors(h, F, x)
    return load().dg_batch_solve(h, int(inner_dtype), int(inner_m), float(inner_tol), int(max_outer), Fp, xp,
                                 *_batch_outputs(its, relres, status, n_inst))


def dg_batch_gmres_ir_solve(h, inner_dtype, inner_m, inner_tol, max_outer, F, x, its=None, relres=None,
                            status=None, n_inst=None):
    Fp, xp = _solve_vectors(h, F, x)
    return load().dg_batch_gmres_ir_solve(h, int(inner_dtype), int(inner_m), float(inner_tol), int(max_outer), Fp,
                                          xp, *_batch_outputs(its, relres, status, n_inst))


def _group_args(hs, F, xs, its, relres, status):
    """Pointer arrays of a group call: handles, and per batch F (device, may be
    None), x (device), its / relres / status (host numpy, may be None)."""
    nh = len(hs)
    P = c_void_p * nh
    harr = P(*[h.value if isinstance(h, c_void_p) else h for h in hs])
    keep = []

    def arr(vals, conv):
        if vals is None:
            return None
        a = P(*[conv(v, i) for i, v in enumerate(vals)])
        keep.append(a)
        return ctypes.cast(a, c_void_p)

    sizes = [_sizes(h) for h in hs]
    dof = lambda i: None if sizes[i] is None else sizes[i].dofs
    Fa = arr(F, lambda v, i: _dev(v, dof(i), "f64", "F"))
    xa = arr(xs, lambda v, i: _dev(v, dof(i), "f64", "x"))
    ia = arr(its, lambda v, i: _host(v, None, "i32", "its"))
    ra = arr(relres, lambda v, i: _host(v, None, "f64", "relres"))
    sa = arr(status, lambda v, i: _host(v, None, "i32", "status"))
    return harr, nh, Fa, xa, ia, ra, sa, keep


def dg_batch_group_solve(hs, inner_dtype, inner_m, inner_tol, max_outer, F, xs, its=None, relres=None, status=None):
    harr, nh, Fa, xa, ia, ra, sa, _keep = _group_args(hs, F, xs, its, relres, status)
    return load().dg_batch_group_solve(ctypes.cast(harr, c_void_p), nh, int(inner_dtype), int(inner_m),
                                       float(inner_tol), int(max_outer), Fa, xa, ia, ra, sa)


def dg_batch_group_gmres_ir_solve(hs, inner_dtype, inner_m, inner_tol, max_outer, F, xs, its=None, relres=None,
                                  status=None):
    harr, nh, Fa, xa, ia, ra, sa, _keep = _group_args(hs, F, xs, its, relres, status)
    return load().dg_batch_group_gmres_ir_solve(ctypes.cast(harr, c_void_p), nh, int(inner_dtype), int(inner_m),
                                                float(inner_tol), int(max_outer), Fa, xa, ia, ra, sa)


def batch_group(dgs, solver="gmres_ir", inner_dtype=DG_F32, inner_m=32, inner_tol=1e-3, max_outer=500,
                raise_on_nonconv=True):
    """Solve the batches of several DG objects (e.g. one per degree) in one
    group call; returns per batch (x, its, relres, status)."""
    xs = [d._empty((d.info().dofs,)) for d in dgs]
    its = [np.zeros(d.batch_n, np.int32) for d in dgs]
    rr = [np.zeros(d.batch_n) for d in dgs]
    st = [np.zeros(d.batch_n, np.int32) for d in dgs]
    fn = dg_batch_group_gmres_ir_solve if solver == "gmres_ir" else dg_batch_group_solve
    s = fn([d.h for d in dgs], inner_dtype, inner_m, inner_tol, max_outer, None, xs, its, rr, st)
    if s != DG_OK and not (s == DG_NOT_CONVERGED and not raise_on_nonconv):
        msgs = "; ".join(dg_last_error(d.h) for d in dgs)
        raise DGError(s, msgs)
    return [(xs[i], its[i], rr[i], st[i]) for i in range(len(dgs))]


def dg_mesh_refine(nodes, elems, dirichlet, neumann):
    """The paper's uniformrefine (Sec. 2.1) through libdg: one red refinement of
    host arrays; returns (nodes, elems, dirichlet, neumann) as numpy arrays."""
    lib = load()
    nodes = np.ascontiguousarray(nodes, dtype=np.float64).reshape(-1, 2)
    elems = np.ascontiguousarray(elems, dtype=np.int32).reshape(-1, 3)
    dirichlet = np.ascontiguousarray(dirichlet, dtype=np.int32).reshape(-1, 2)
    neumann = np.ascontiguousarray(neumann, dtype=np.int32).reshape(-1, 2)
    sizes = [ctypes.c_int() for _ in range(4)]
    args = (_host(nodes), nodes.shape[0], _host(elems), elems.shape[0], _host(dirichlet), dirichlet.shape[0],
            _host(neumann), neumann.shape[0])
    s = lib.dg_mesh_refine(*args, None, ctypes.byref(sizes[0]), None, ctypes.byref(sizes[1]), None,
                           ctypes.byref(sizes[2]), None, ctypes.byref(sizes[3]))
    if s != DG_OK:
        raise DGError(s, "dg_mesh_refine")
    nv, ne, nd, nn = (v.value for v in sizes)
    out = (np.zeros((nv, 2)), np.zeros((ne, 3), np.int32), np.zeros((nd, 2), np.int32), np.zeros((nn, 2), np.int32))
    s = lib.dg_mesh_refine(*args, _host(out[0]), ctypes.byref(sizes[0]), _host(out[1]), ctypes.byref(sizes[1]),
                           _host(out[2]), ctypes.byref(sizes[2]), _host(out[3]), ctypes.byref(sizes[3]))
    if s != DG_OK:
        raise DGError(s, "dg_mesh_refine")
    return out


def dg_nonlinear_global(h, p, c, x, H, HJ=None):
    i = _sizes(h)
    n = None if i is None else i.dofs
    return load().dg_nonlinear_global(h, int(p), float(c), _dev(x, n, "f64", "x"), _dev(H, n, "f64", "H"),
                                      _dev(HJ, None if i is None else i.ne * i.nb * i.nb, "f64", "HJ"))


def dg_newton_solve(h, p, c, max_newton, lin_tol, F, x, info):
    Fp, xp = _solve_vectors(h, F, x)
    return load().dg_newton_solve(h, int(p), float(c), int(max_newton), float(lin_tol), Fp, xp,
                                  ctypes.byref(info))


def dg_mlp_num_params(degree):
    n = c_int64()
    s = load().dg_mlp_num_params(int(degree), ctypes.byref(n))
    if s != DG_OK:
        raise DGError(s, "dg_mlp_num_params")
    return n.value


def dg_mlp_init(h, seed):
    return load().dg_mlp_init(h, int(seed))


def dg_mlp_set_weights(h, theta):
    theta = np.ascontiguousarray(theta, dtype=np.float32)
    return load().dg_mlp_set_weights(h, _host(theta), theta.size)


def dg_mlp_get_weights(h, n):
    out = np.zeros(n, np.float32)
    s = load().dg_mlp_get_weights(h, _host(out), n)
    return s, out


def dg_mlp_collect(h, F, xk):
    Fp, xp = _solve_vectors(h, F, xk)
    return load().dg_mlp_collect(h, Fp, xp)


def dg_mlp_collect_basis(h, nvec):
    return load().dg_mlp_collect_basis(h, int(nvec))


def dg_mlp_num_rows(h):
    n = c_int64()
    s = load().dg_mlp_num_rows(h, ctypes.byref(n))
    return s, n.value


def _mlp_widths(h):
    i = _sizes(h)
    return (None, None) if i is None else (4 * i.nb + 8, i.nb)


def dg_mlp_get_rows(h, X, T, max_rows):
    din, nb = _mlp_widths(h)
    m = int(max_rows)
    return load().dg_mlp_get_rows(h, _host(X, None if din is None else m * din, "f32", "X"),
                                  _host(T, None if nb is None else m * nb, "f32", "T"), m)


def dg_mlp_clear_data(h):
    return load().dg_mlp_clear_data(h)


def dg_mlp_train(h, steps, batch_rows, lr, seed, loss=None):
    return load().dg_mlp_train(h, int(steps), int(batch_rows), float(lr), int(seed),
                               _host(loss, int(steps), "f32", "loss"))


def dg_mlp_loss_grad(h, X, T, rows, grad=None):
    loss = c_double()
    din, nb = _mlp_widths(h)
    r = int(rows)
    s = load().dg_mlp_loss_grad(h, _dev(X, None if din is None else r * din, "f32", "X"),
                                _dev(T, None if nb is None else r * nb, "f32", "T"), r, ctypes.byref(loss),
                                _host(grad, None, "f32", "grad"))
    return s, loss.value


def dg_mlp_forward(h, X, rows, Y):
    din, nb = _mlp_widths(h)
    r = int(rows)
    return load().dg_mlp_forward(h, _dev(X, None if din is None else r * din, "f32", "X"), r,
                                 _dev(Y, None if nb is None else r * nb, "f32", "Y"))


def dg_get_launch_count(h):
    c = c_int64()
    s = load().dg_get_launch_count(h, ctypes.byref(c))
    return s, c.value


def dg_reference_basis(degree, rs):
    rs = np.ascontiguousarray(rs, dtype=np.float64).reshape(-1, 2)
    nb = (degree + 1) * (degree + 2) // 2
    phi = np.zeros((rs.shape[0], nb)); dr = np.zeros_like(phi); ds = np.zeros_like(phi)
    s = load().dg_reference_basis(int(degree), rs.shape[0], _host(rs), _host(phi), _host(dr), _host(ds))
    if s != DG_OK:
        raise DGError(s, "dg_reference_basis")
    return phi, dr, ds


def dg_reference_rule(which, degree):
    n = ctypes.c_int()
    load().dg_reference_rule(int(which), int(degree), None, None, ctypes.byref(n))
    rs = np.zeros((n.value, 2)); w = np.zeros(n.value)
    s = load().dg_reference_rule(int(which), int(degree), _host(rs), _host(w), ctypes.byref(n))
    if s != DG_OK:
        raise DGError(s, "dg_reference_rule")
    return rs, w


# ---------------------------------------------------------------------------
# object wrapper
# ---------------------------------------------------------------------------
class DG:
    """One libdg handle on a CUDA device; work goes to torch's current stream."""

    def __init__(self, device: int = 0, stream=None):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", device)
        self._own_stream = None
        if stream is None:
            cur = torch.cuda.current_stream(self.device)
            if cur.cuda_stream == 0:
                # the legacy default stream cannot be captured into CUDA graphs:
                # use a stream of our own that is ordered with the legacy one
                self._own_stream = dg_stream_create(device)
                stream = self._own_stream
            else:
                stream = cur.cuda_stream
        self.h = dg_create(device, stream)
        self.params = dg_params_default()
        self._memory_source = None

    def close(self):
        if self.h is not None:
            dg_destroy(self.h)
            self.h = None
        self._memory_source = None
        if self._own_stream is not None:
            dg_stream_destroy(self._own_stream)
            self._own_stream = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, s):
        if s != DG_OK:
            raise DGError(s, dg_last_error(self.h))

    # -- device memory --------------------------------------------------------
    def set_arena(self, buf):
        """Carve the handle's device memory out of `buf` (a CUDA tensor the
        object keeps alive); right after construction only."""
        self.check(dg_set_arena(self.h, buf, buf.numel() * buf.element_size()))
        self._memory_source = buf

    def use_torch_allocator(self):
        """Take the handle's device memory from torch's caching allocator
        (counted by torch.cuda.memory_allocated); right after construction only."""
        torch = self.torch

        def alloc(ctx, nbytes, device, stream):
            return torch.cuda.caching_allocator_alloc(int(nbytes), device=int(device), stream=int(stream or 0))

        def free(ctx, ptr, nbytes, device, stream):
            torch.cuda.caching_allocator_delete(int(ptr))

        fns = (DG_ALLOC_FN(alloc), DG_FREE_FN(free))
        self.check(dg_set_allocator(self.h, *fns))
        self._memory_source = fns

    def workspace_size(self, what=DG_WS_TOTAL):
        return dg_workspace_size(self.h, what)

    # -- set-up -------------------------------------------------------------
    def mesh_upload(self, nodes, elems, dirichlet, neumann):
        self.check(dg_mesh_upload(self.h, nodes, elems, dirichlet, neumann))

    def set_params(self, **kw):
        for k, v in kw.items():
            setattr(self.params, k, v)
        self.check(dg_set_params(self.h, self.params))

    def info(self):
        s, i = dg_get_info(self.h)
        self.check(s)
        return i

    def _empty(self, shape, dtype=None):
        return self.torch.empty(shape, dtype=dtype or self.torch.float64, device=self.device)

    def quad_points(self, which):
        i = self.info()
        shape = {DG_POINTS_VOLUME: (i.ne, i.q_volume, 2), DG_POINTS_BOUNDARY: (i.n_bedges, i.q_edge, 2),
                 DG_POINTS_ERROR: (i.ne, i.q_error, 2), DG_POINTS_FACE: (i.ne, 3, i.q_edge, 2)}[which]
        out = self._empty(shape)
        self.check(dg_quad_points(self.h, which, out))
        return out

    def boundary_info(self):
        i = self.info()
        n = self._empty((i.n_bedges, 2))
        t = self._empty((i.n_bedges,), self.torch.int32)
        self.check(dg_boundary_info(self.h, n, t))
        return n, t

    def assemble(self, eps, alpha, b, f=None, gD=None, gN=None, f_const=0.0, gD_const=0.0, gN_const=0.0,
                 eps_q=None, eps_f=None):
        """eps_q / eps_f: a pointwise diffusion coefficient at DG_POINTS_VOLUME
        and DG_POINTS_FACE (then eps is not used), or None for the constant eps."""
        c = dg_coeffs()
        c.eps, c.alpha = float(eps), float(alpha)
        for t in range(6):
            c.b[t] = float(b[t])
        self._keep = (f, gD, gN, eps_q, eps_f)
        dg_coeffs_data(self.h, c, f, gD, gN, eps_q, eps_f)
        c.f_const, c.gD_const, c.gN_const = float(f_const), float(gD_const), float(gN_const)
        self.check(dg_assemble(self.h, c))

    def rhs(self):
        i = self.info()
        F = self._empty((i.dofs,))
        self.check(dg_get_rhs(self.h, F))
        return F

    def blocks(self, dtype=DG_F64):
        import torch
        i = self.info()
        td = {DG_F64: torch.float64, DG_F32: torch.float32, DG_BF16: torch.bfloat16}[dtype]
        out = self._empty((i.ne, 4, i.nb, i.nb), td)
        nbr = self._empty((i.ne, 3), torch.int32)
        self.check(dg_get_blocks(self.h, dtype, out, nbr))
        return out, nbr

    # -- operators ------------------------------------------------------------
    def apply(self, x, dtype=DG_F64, y=None):
        y = self.torch.empty_like(x) if y is None else y
        self.check(dg_apply(self.h, dtype, x, y))
        return y

    def precond_setup(self, kind=DG_PRECOND_BLOCK_JACOBI):
        self.check(dg_precond_setup(self.h, kind))

    def precond_apply(self, r, dtype=DG_F64, z=None):
        z = self.torch.empty_like(r) if z is None else z
        self.check(dg_precond_apply(self.h, dtype, r, z))
        return z

    # -- solvers --------------------------------------------------------------
    def gmres_solve(self, F=None, x=None, raise_on_nonconv=True):
        i = self.info()
        x = self._empty((i.dofs,)) if x is None else x
        info = dg_solve_info()
        s = dg_gmres_solve(self.h, F, x, info)
        if s != DG_OK and not (s == DG_NOT_CONVERGED and not raise_on_nonconv):
            self.check(s)
        return x, info

    def mixed_solve(self, inner_dtype=DG_BF16, inner_m=30, inner_tol=1e-3, max_outer=30, F=None, x=None,
                    raise_on_nonconv=True):
        i = self.info()
        x = self._empty((i.dofs,)) if x is None else x
        info = dg_solve_info()
        s = dg_mixed_solve(self.h, inner_dtype, inner_m, inner_tol, max_outer, F, x, info)
        if s != DG_OK and not (s == DG_NOT_CONVERGED and not raise_on_nonconv):
            self.check(s)
        return x, info

    def gmres_ir_solve(self, inner_dtype=DG_BF16, inner_m=50, inner_tol=1e-2, max_outer=200, F=None, x=None,
                       raise_on_nonconv=True):
        i = self.info()
        x = self._empty((i.dofs,)) if x is None else x
        info = dg_solve_info()
        s = dg_gmres_ir_solve(self.h, inner_dtype, inner_m, inner_tol, max_outer, F, x, info)
        if s != DG_OK and not (s == DG_NOT_CONVERGED and not raise_on_nonconv):
            self.check(s)
        return x, info

    def nonlinear_global(self, x, p=2, c=1.0, want_jacobian=True):
        """H(x) [dofs] and, if asked, the element blocks of its Jacobian [ne, nb, nb]."""
        i = self.info()
        nb = i.dofs // i.ne
        H = self._empty((i.dofs,))
        HJ = self._empty((i.ne, nb, nb)) if want_jacobian else None
        self.check(dg_nonlinear_global(self.h, p, c, x, H, HJ))
        return H, HJ

    def newton_solve(self, p=2, c=1.0, max_newton=50, lin_tol=1e-12, F=None, x=None, raise_on_nonconv=True):
        i = self.info()
        x = self._empty((i.dofs,)) if x is None else x
        info = dg_solve_info()
        s = dg_newton_solve(self.h, p, c, max_newton, lin_tol, F, x, info)
        if s != DG_OK and not (s == DG_NOT_CONVERGED and not raise_on_nonconv):
            self.check(s)
        return x, info

    def dense_solve(self, F=None):
        i = self.info()
        x = self._empty((i.dofs,))
        self.check(dg_dense_solve(self.h, F, x))
        return x

    def l2_error(self, x, uex_q):
        s, l2, hmax = dg_l2_error(self.h, x, uex_q)
        self.check(s)
        return l2, hmax

    def profile_kernel(self, which, dtype, j, reps=20):
        s, ms = dg_profile_kernel(self.h, which, dtype, j, reps)
        self.check(s)
        return ms

    def batch_setup(self, elem_start, coeffs):
        self.check(dg_batch_setup(self.h, elem_start, coeffs))
        self.batch_n = len(elem_start) - 1

    def batch_clear(self):
        self.check(dg_batch_clear(self.h))

    def batch_autotune(self):
        s, t = dg_batch_autotune(self.h)
        self.check(s)
        return t

    def batch_solve(self, inner_dtype=DG_F32, inner_m=30, inner_tol=1e-4, max_outer=30, F=None, x=None,
                    raise_on_nonconv=True):
        i = self.info()
        x = self._empty((i.dofs,)) if x is None else x
        n = self.batch_n
        its = np.zeros(n, np.int32); rr = np.zeros(n); st = np.zeros(n, np.int32)
        s = dg_batch_solve(self.h, inner_dtype, inner_m, inner_tol, max_outer, F, x, its, rr, st, n_inst=n)
        if s != DG_OK and not (s == DG_NOT_CONVERGED and not raise_on_nonconv):
            self.check(s)
        return x, its, rr, st

    def batch_gmres_ir_solve(self, inner_dtype=DG_F32, inner_m=32, inner_tol=1e-3, max_outer=500, F=None, x=None,
                             raise_on_nonconv=True):
        i = self.info()
        x = self._empty((i.dofs,)) if x is None else x
        n = self.batch_n
        its = np.zeros(n, np.int32); rr = np.zeros(n); st = np.zeros(n, np.int32)
        s = dg_batch_gmres_ir_solve(self.h, inner_dtype, inner_m, inner_tol, max_outer, F, x, its, rr, st,
                                    n_inst=n)
        if s != DG_OK and not (s == DG_NOT_CONVERGED and not raise_on_nonconv):
            self.check(s)
        return x, its, rr, st

    # -- learned preconditioner -------------------------------------------------
    def mlp_init(self, seed=0):
        self.check(dg_mlp_init(self.h, seed))

    def mlp_set_weights(self, theta):
        self.check(dg_mlp_set_weights(self.h, theta))

    def mlp_get_weights(self):
        s, th = dg_mlp_get_weights(self.h, dg_mlp_num_params(self.params.degree))
        self.check(s)
        return th

    def mlp_collect(self, xk, F=None):
        self.check(dg_mlp_collect(self.h, F, xk))

    def mlp_collect_basis(self, nvec):
        self.check(dg_mlp_collect_basis(self.h, nvec))

    def mlp_rows(self):
        s, n = dg_mlp_num_rows(self.h)
        self.check(s)
        return n

    def mlp_train(self, steps, batch_rows=4096, lr=1e-3, seed=0):
        loss = np.zeros(steps, np.float32)
        self.check(dg_mlp_train(self.h, steps, batch_rows, lr, seed, loss))
        return loss

    def launch_count(self):
        s, c = dg_get_launch_count(self.h)
        self.check(s)
        return c

    def eval(self, x, rs):
        rs = np.ascontiguousarray(rs, dtype=np.float64).reshape(-1, 2)
        out = self._empty((self.info().ne, rs.shape[0]))
        self.check(dg_eval(self.h, x, rs, out))
        return out

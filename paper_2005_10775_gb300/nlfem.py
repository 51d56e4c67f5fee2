"""ctypes binding of libnlfem (include/nlfem.h): argument marshalling only.

Every function keeps the C name and forwards to the library; all of the
method's work runs in the library's CUDA kernels.  Arrays may be numpy arrays
(host memory) or CUDA torch tensors (device memory).  Importing this module
loads the in-tree library and fails loudly if it has not been built.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libnlfem.so")

NL_OK, NL_EINVAL, NL_ENOMEM, NL_ECUDA, NL_EGEOM, NL_ETIMEOUT, NL_ENOCONV, NL_EUNSUPPORTED = range(8)
BALL = {"barycenter": 0, "nocaps": 1, "approxcaps": 2, "exactcaps": 3, "ngon": 4, "overlap": 5,
        "bary_nocaps": 6, "bary_approxcaps": 7}
RULE = {"gauss3": 0, "gauss4": 1, "paper7": 2, "dunavant7": 3, "dunavant16": 4, "switch47": 5}
KERNEL = {"const": 0, "inv_dist": 1}
PREC = {"fp64": 0, "fp32c": 1}


class NlError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"libnlfem status {status}: {msg}")
        self.status = status


class nl_mesh(ctypes.Structure):
    _fields_ = [("nv", ctypes.c_int32), ("nt", ctypes.c_int32),
                ("vx", ctypes.c_void_p), ("vy", ctypes.c_void_p), ("tri", ctypes.c_void_p),
                ("node_in_omega", ctypes.c_void_p), ("elem_in_omega", ctypes.c_void_p)]


class nl_config(ctypes.Structure):
    _fields_ = [("delta", ctypes.c_double), ("kernel_c", ctypes.c_double),
                ("kernel", ctypes.c_int32), ("ball", ctypes.c_int32), ("ngon_n", ctypes.c_int32),
                ("cap_m", ctypes.c_int32), ("ngon_offsets", ctypes.c_void_p),
                ("outer", ctypes.c_int32), ("inner", ctypes.c_int32), ("prec", ctypes.c_int32),
                ("duffy_n", ctypes.c_int32), ("cap_printed", ctypes.c_int32), ("shifted", ctypes.c_int32)]


class nl_csr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nnz", ctypes.c_int64), ("row_ptr", ctypes.c_void_p),
                ("col_idx", ctypes.c_void_p), ("val", ctypes.c_void_p), ("n_pairs", ctypes.c_int64),
                ("n_qp_pairs", ctypes.c_int64), ("n_inter", ctypes.c_int64), ("priv", ctypes.c_void_p)]


class nl_batch_info(ctypes.Structure):
    _fields_ = [("chunk", ctypes.c_int32), ("order", ctypes.c_int32), ("blocks", ctypes.c_int32),
                ("launches", ctypes.c_int32), ("source", ctypes.c_int32), ("n_tried", ctypes.c_int32),
                ("tuned_ms", ctypes.c_double), ("default_ms", ctypes.c_double),
                ("mode", ctypes.c_int32), ("streams", ctypes.c_int32)]


NL_BATCH_NO_TUNE = 1
NL_BATCH_PER_PROBLEM = 2
SCHED_SOURCES = {0: "default", 1: "tuned", 2: "cached"}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                          "(python -m paper_2005_10775_gb300.build); there is no CPU fallback")
    L = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    sig = {
        "nl_create": (ctypes.c_int, [P(ctypes.c_void_p), ctypes.c_int, ctypes.c_void_p]),
        "nl_destroy": (None, [ctypes.c_void_p]),
        "nl_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
        "nl_assemble": (ctypes.c_int, [ctypes.c_void_p, P(nl_mesh), P(nl_config), P(nl_csr)]),
        "nl_assemble_numeric": (ctypes.c_int, [ctypes.c_void_p, P(nl_csr)]),
        "nl_assemble_batch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, P(nl_mesh), P(nl_config),
                                             P(nl_csr)]),
        "nl_batch_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, P(nl_mesh), P(nl_config), P(nl_csr),
                                           ctypes.c_int32, P(ctypes.c_void_p)]),
        "nl_batch_run": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
        "nl_batch_get_info": (ctypes.c_int, [ctypes.c_void_p, P(nl_batch_info)]),
        "nl_batch_destroy": (None, [ctypes.c_void_p, ctypes.c_void_p]),
        "nl_interactions": (ctypes.c_int, [ctypes.c_void_p, P(nl_mesh), P(nl_config), ctypes.c_void_p,
                                           ctypes.c_void_p, ctypes.c_void_p]),
        "nl_extract": (ctypes.c_int, [ctypes.c_void_p, P(nl_csr), P(nl_mesh), P(nl_csr), P(nl_csr)]),
        "nl_rhs": (ctypes.c_int, [ctypes.c_void_p, P(nl_csr), P(nl_mesh), ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_void_p]),
        "nl_matvec": (ctypes.c_int, [ctypes.c_void_p, P(nl_csr), ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_int32]),
        "nl_cg": (ctypes.c_int, [ctypes.c_void_p, P(nl_csr), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                 ctypes.c_int32, P(ctypes.c_int32), P(ctypes.c_double)]),
        "nl_csr_download": (ctypes.c_int, [ctypes.c_void_p, P(nl_csr), ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p]),
        "nl_csr_free": (None, [ctypes.c_void_p, P(nl_csr)]),
        "nl_last_timings": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
        "nl_launch_count": (ctypes.c_int64, [ctypes.c_void_p]),
        "nl_fma_peak": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, P(ctypes.c_double)]),
        "nl_last_fp64_items": (ctypes.c_int64, [ctypes.c_void_p]),
        "nl_cg_noalloc": (ctypes.c_int, [ctypes.c_void_p, P(nl_csr), ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_double, ctypes.c_int32, P(ctypes.c_int32), P(ctypes.c_double)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


_L = _load()
LIB = _L


class _Keep(list):
    """Keeps marshalled arrays alive for the duration of a call."""


def _ptr(a, keep, dtype=None):
    """Data pointer of a numpy array (host) or torch tensor (host or CUDA)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr") and hasattr(a, "is_cuda"):
        if dtype is not None:
            import torch
            tdt = {np.float64: torch.float64, np.int32: torch.int32, np.uint8: torch.uint8}[dtype]
            if a.dtype != tdt:
                a = a.to(tdt)
        a = a.contiguous()
        keep.append(a)
        return a.data_ptr()
    a = np.ascontiguousarray(a, dtype=dtype) if dtype is not None else np.ascontiguousarray(a)
    keep.append(a)
    return a.ctypes.data


def _out_ptr(a, n, keep, what, device=None):
    """Data pointer of an output (or in/out) float64 vector of n entries, written in place.
    It is never cast or copied (a copy would lose the result), so a wrong dtype, a
    non-contiguous array, a wrong length or a CUDA tensor on another device than the
    context's is rejected with NlError(NL_EINVAL) before anything is launched."""
    if hasattr(a, "data_ptr") and hasattr(a, "is_cuda"):
        import torch
        if a.dtype != torch.float64:
            raise NlError(NL_EINVAL, f"{what} must be float64 (got {a.dtype})")
        if not a.is_contiguous():
            raise NlError(NL_EINVAL, f"{what} must be contiguous")
        if a.numel() != n:
            raise NlError(NL_EINVAL, f"{what} must hold {n} entries (got {a.numel()})")
        if device is not None and a.is_cuda and a.device.index != device:
            raise NlError(NL_EINVAL, f"{what} is on cuda:{a.device.index}, the context on cuda:{device}")
        keep.append(a)
        return a.data_ptr()
    if not isinstance(a, np.ndarray):
        raise NlError(NL_EINVAL, f"{what} must be a numpy array or a torch tensor")
    if a.dtype != np.float64:
        raise NlError(NL_EINVAL, f"{what} must be float64 (got {a.dtype})")
    if not a.flags.c_contiguous or not a.flags.writeable:
        raise NlError(NL_EINVAL, f"{what} must be contiguous and writeable")
    if a.size != n:
        raise NlError(NL_EINVAL, f"{what} must hold {n} entries (got {a.size})")
    keep.append(a)
    return a.ctypes.data


def _in_vec(a, n, keep, what):
    """Data pointer of an input float64 vector of n entries (host arrays of another dtype are
    converted; the length is checked, so the library never reads past the end)."""
    size = a.numel() if hasattr(a, "numel") else np.asarray(a).size
    if size != n:
        raise NlError(NL_EINVAL, f"{what} must hold {n} entries (got {size})")
    return _ptr(a, keep, np.float64)


# device of each context created through this binding (checks of CUDA tensors)
_CTX_DEVICE = {}


def _check(ctx, st):
    if st != NL_OK:
        raise NlError(st, _L.nl_last_error(ctx).decode(errors="replace"))


def make_mesh(mesh, keep) -> nl_mesh:
    """nl_mesh from an object with vx, vy, tri and optional node/elem labels."""
    tri = mesh.tri
    nt = int(tri.shape[0]) if getattr(tri, "ndim", 1) == 2 else int(tri.shape[0]) // 3
    vx = mesh.vx
    return nl_mesh(int(vx.shape[0]), nt, _ptr(vx, keep, np.float64), _ptr(mesh.vy, keep, np.float64),
                   _ptr(tri, keep, np.int32),
                   _ptr(getattr(mesh, "node_in_omega", None), keep, np.uint8),
                   _ptr(getattr(mesh, "elem_in_omega", None), keep, np.uint8))


def make_config(keep, delta, ball, outer="dunavant7", inner="dunavant7", kernel="const", kernel_c=1.0,
                ngon_off=None, cap_m=2, prec="fp64", duffy_n=4, cap_printed=0, shifted=0) -> nl_config:
    n = 0 if ngon_off is None else int(ngon_off.shape[0])
    return nl_config(float(delta), float(kernel_c), KERNEL[kernel], BALL[ball], n, int(cap_m),
                     _ptr(ngon_off, keep, np.float64), RULE[outer], RULE[inner], PREC[prec], int(duffy_n),
                     int(cap_printed), int(shifted))


def config_of(problem, keep, **over) -> nl_config:
    kw = dict(delta=problem.delta, ball=problem.ball, outer=problem.outer, inner=problem.inner,
              kernel=problem.kernel, kernel_c=problem.kernel_c, ngon_off=problem.ngon_off, cap_m=problem.cap_m)
    kw.update(over)
    return make_config(keep, **kw)


# ---------------------------------------------------------------------------
# the C entry points
# ---------------------------------------------------------------------------

def nl_create(device: int = 0, stream: int | None = None):
    h = ctypes.c_void_p()
    st = _L.nl_create(ctypes.byref(h), int(device), ctypes.c_void_p(stream) if stream else None)
    if st != NL_OK:
        raise NlError(st, "nl_create failed")
    _CTX_DEVICE[h.value] = int(device)
    return h


def nl_destroy(ctx):
    _CTX_DEVICE.pop(getattr(ctx, "value", None), None)
    _L.nl_destroy(ctx)


def nl_last_error(ctx) -> str:
    return _L.nl_last_error(ctx).decode(errors="replace")


def nl_assemble(ctx, mesh: nl_mesh, cfg: nl_config) -> nl_csr:
    out = nl_csr()
    _check(ctx, _L.nl_assemble(ctx, ctypes.byref(mesh), ctypes.byref(cfg), ctypes.byref(out)))
    return out


def nl_assemble_numeric(ctx, m: nl_csr) -> None:
    _check(ctx, _L.nl_assemble_numeric(ctx, ctypes.byref(m)))


def nl_assemble_batch(ctx, meshes, cfgs):
    n = len(meshes)
    M = (nl_mesh * n)(*meshes)
    C = (nl_config * n)(*cfgs)
    O = (nl_csr * n)()
    _check(ctx, _L.nl_assemble_batch(ctx, n, M, C, O))
    return list(O)


def nl_batch_create(ctx, meshes, cfgs, flags: int = 0):
    """Returns (handle, [nl_csr] * n); the matrices stay valid after nl_batch_destroy
    and are freed with nl_csr_free."""
    n = len(meshes)
    M = (nl_mesh * n)(*meshes)
    C = (nl_config * n)(*cfgs)
    O = (nl_csr * n)()
    h = ctypes.c_void_p()
    _check(ctx, _L.nl_batch_create(ctx, n, M, C, O, flags, ctypes.byref(h)))
    return h, list(O)


def nl_batch_run(ctx, batch) -> None:
    _check(ctx, _L.nl_batch_run(ctx, batch))


def nl_batch_get_info(batch) -> dict:
    info = nl_batch_info()
    st = _L.nl_batch_get_info(batch, ctypes.byref(info))
    if st != NL_OK:
        raise NlError(st, "nl_batch_get_info")
    d = {k: getattr(info, k) for k, _ in nl_batch_info._fields_}
    d["source"] = SCHED_SOURCES.get(d["source"], str(d["source"]))
    return d


def nl_batch_destroy(ctx, batch) -> None:
    _L.nl_batch_destroy(ctx, batch)


def nl_interactions(ctx, mesh: nl_mesh, cfg: nl_config):
    K = mesh.nt
    h = np.zeros(K, np.uint64)
    c = np.zeros(K, np.int64)
    q = np.zeros(K, np.int64)
    _check(ctx, _L.nl_interactions(ctx, ctypes.byref(mesh), ctypes.byref(cfg), h.ctypes.data, c.ctypes.data,
                                   q.ctypes.data))
    return h, c, q


def nl_extract(ctx, D: nl_csr, mesh: nl_mesh):
    A, B = nl_csr(), nl_csr()
    _check(ctx, _L.nl_extract(ctx, ctypes.byref(D), ctypes.byref(mesh), ctypes.byref(A), ctypes.byref(B)))
    B._rect = True   # its columns are the Omega_I nodes (the library holds their count)
    return A, B


def nl_rhs(ctx, B: nl_csr, mesh: nl_mesh, f_nodal, g_nodal, F=None):
    keep = _Keep()
    if F is None:
        F = np.zeros(B.n)
    dev = _CTX_DEVICE.get(getattr(ctx, "value", None))
    _check(ctx, _L.nl_rhs(ctx, ctypes.byref(B), ctypes.byref(mesh), _in_vec(f_nodal, mesh.nv, keep, "f_nodal"),
                          _in_vec(g_nodal, mesh.nv, keep, "g_nodal"), _out_ptr(F, B.n, keep, "F", dev)))
    return F


def nl_matvec(ctx, A: nl_csr, x, y=None, prec="fp64"):
    keep = _Keep()
    if y is None:
        y = np.zeros(A.n)
    dev = _CTX_DEVICE.get(getattr(ctx, "value", None))
    # a square A takes n entries of x; the rectangular B of nl_extract one per Omega_I node
    xp = _ptr(x, keep, np.float64) if getattr(A, "_rect", False) else _in_vec(x, A.n, keep, "x")
    _check(ctx, _L.nl_matvec(ctx, ctypes.byref(A), xp, _out_ptr(y, A.n, keep, "y", dev), PREC[prec]))
    return y


def nl_cg(ctx, A: nl_csr, b, x, rtol=1e-10, max_it=10000):
    """x holds the initial guess and receives the solution in place (numpy array or tensor)."""
    keep = _Keep()
    it = ctypes.c_int32()
    rr = ctypes.c_double()
    dev = _CTX_DEVICE.get(getattr(ctx, "value", None))
    _check(ctx, _L.nl_cg(ctx, ctypes.byref(A), _in_vec(b, A.n, keep, "b"), _out_ptr(x, A.n, keep, "x", dev),
                         float(rtol), int(max_it), ctypes.byref(it), ctypes.byref(rr)))
    return int(it.value), float(rr.value)


def nl_cg_noalloc(ctx, A: nl_csr, b, x, rtol=1e-10, max_it=10000):
    """b and x must be contiguous float64 CUDA tensors of A.n entries on the context's device;
    x holds the initial guess and is updated in place.  Anything else is rejected with
    NlError(NL_EINVAL) before the library is called (no cast, no copy)."""
    keep = _Keep()
    it = ctypes.c_int32()
    rr = ctypes.c_double()
    dev = _CTX_DEVICE.get(getattr(ctx, "value", None))
    bp = _out_ptr(b, A.n, keep, "b", dev)   # read only, but held to the same rules: no copy of a device vector
    xp = _out_ptr(x, A.n, keep, "x", dev)
    for v, name in ((b, "b"), (x, "x")):
        if not getattr(v, "is_cuda", False):
            raise NlError(NL_EINVAL, f"nl_cg_noalloc needs {name} in device memory (a CUDA tensor)")
    _check(ctx, _L.nl_cg_noalloc(ctx, ctypes.byref(A), bp, xp, float(rtol), int(max_it),
                                 ctypes.byref(it), ctypes.byref(rr)))
    return int(it.value), float(rr.value)


def nl_csr_download(ctx, m: nl_csr):
    rp = np.zeros(m.n + 1, np.int64)
    ci = np.zeros(max(m.nnz, 1), np.int32)
    va = np.zeros(max(m.nnz, 1), np.float64)
    _check(ctx, _L.nl_csr_download(ctx, ctypes.byref(m), rp.ctypes.data, ci.ctypes.data, va.ctypes.data))
    return rp, ci[:m.nnz], va[:m.nnz]


def nl_csr_free(ctx, m: nl_csr):
    _L.nl_csr_free(ctx, ctypes.byref(m))


def nl_last_timings(ctx):
    t = np.zeros(4)
    _check(ctx, _L.nl_last_timings(ctx, t.ctypes.data))
    return t


def nl_fma_peak(ctx, prec="fp32c") -> float:
    """Measured FMA throughput of the context's GPU in TFLOP/s (FP32 for "fp32c", FP64 for "fp64")."""
    t = ctypes.c_double()
    _check(ctx, _L.nl_fma_peak(ctx, PREC[prec], ctypes.byref(t)))
    return float(t.value)


def nl_launch_count(ctx) -> int:
    return int(_L.nl_launch_count(ctx))


def nl_last_fp64_items(ctx) -> int:
    """Items of the last FP32-path nl_assemble / nl_interactions whose region the FP64
    geometry built (queued for the deferred kernel, or inline when the queue was full)."""
    return int(_L.nl_last_fp64_items(ctx))


def to_scipy(ctx, m: nl_csr, ncols=None):
    import scipy.sparse as sp
    rp, ci, va = nl_csr_download(ctx, m)
    return sp.csr_matrix((va, ci, rp), shape=(m.n, m.n if ncols is None else ncols))

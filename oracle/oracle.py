"""Python face of the FP64 CPU oracle (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import
this module.  It wraps the plain C oracle (oracle/nl_oracle.c) with ctypes and
adds the numpy/scipy steps of the solve:

  * load vector G_j = int_Omega f phi_j with f given at the nodes (P1 interpolant,
    exact for the linear f of Sec. 8) over elements labelled Omega;
  * F = G - D[Omega, Omega_I] g (Sec. 7.2, assignment rules B and C; the
    Dirichlet volume constraint of Eq. (prob) enters through the nodal
    interpolant of g, Eq. (appr));
  * A U = F solved directly (scipy.sparse.linalg.spsolve);
  * the L2(Omega) error of u_h against a given u (degree-8 rule per element).

It imports nothing from the CUDA package: meshes and problems are passed in as
plain arrays or duck-typed objects (attributes vx, vy, tri, node_in_omega, ...).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "nl_oracle.c")
SO = os.path.join(HERE, "_build", "libnl_oracle.so")

BALL = {"barycenter": 0, "nocaps": 1, "approxcaps": 2, "exactcaps": 3, "ngon": 4, "overlap": 5,
        "bary_nocaps": 6, "bary_approxcaps": 7}
RULE = {"gauss3": 0, "gauss4": 1, "paper7": 2, "dunavant7": 3, "dunavant16": 4, "switch47": 5}
KERNEL = {"const": 0, "inv_dist": 1}
KIND_NONE, KIND_WHOLE, KIND_PARTIAL = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle: plain C, -O2, no FMA contraction, no fast-math, OpenMP."""
    os.makedirs(os.path.dirname(SO), exist_ok=True)
    if force or not os.path.exists(SO) or os.path.getmtime(SO) < os.path.getmtime(SRC):
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
               "-shared", "-o", SO + ".tmp", SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(SO + ".tmp", SO)
    return SO


class _Mesh(ctypes.Structure):
    _fields_ = [("nv", ctypes.c_int32), ("nt", ctypes.c_int32),
                ("vx", ctypes.POINTER(ctypes.c_double)), ("vy", ctypes.POINTER(ctypes.c_double)),
                ("tri", ctypes.POINTER(ctypes.c_int32))]


class _Cfg(ctypes.Structure):
    _fields_ = [("delta", ctypes.c_double), ("kernel_c", ctypes.c_double),
                ("kernel", ctypes.c_int32), ("ball", ctypes.c_int32),
                ("ngon_n", ctypes.c_int32), ("cap_m", ctypes.c_int32),
                ("ngon_off", ctypes.POINTER(ctypes.c_double)),
                ("outer", ctypes.c_int32), ("inner", ctypes.c_int32),
                ("duffy_n", ctypes.c_int32), ("cap_printed", ctypes.c_int32), ("shifted", ctypes.c_int32)]


class _Rec(ctypes.Structure):
    _fields_ = [("a", ctypes.c_int32), ("b", ctypes.c_int32), ("q", ctypes.c_int8),
                ("kind", ctypes.c_int8), ("nverts", ctypes.c_int8), ("ncaps", ctypes.c_int8)]


class _Res(ctypes.Structure):
    _fields_ = [("nnz", ctypes.c_int64), ("row", ctypes.POINTER(ctypes.c_int32)),
                ("col", ctypes.POINTER(ctypes.c_int32)), ("val", ctypes.POINTER(ctypes.c_double)),
                ("n_pairs", ctypes.c_int64), ("n_qp_pairs", ctypes.c_int64), ("n_inter", ctypes.c_int64),
                ("rec", ctypes.POINTER(_Rec)), ("hash_a", ctypes.POINTER(ctypes.c_uint64)),
                ("count_a", ctypes.POINTER(ctypes.c_int64)), ("qp_a", ctypes.POINTER(ctypes.c_int64))]


_LIB = None


def lib():
    global _LIB
    if _LIB is None:
        build()
        _LIB = load(SO)
    return _LIB


def load(path: str):
    """The oracle library at `path` with its entry points typed (lib() loads the built one;
    a test may load a copy compiled with a planted mistake)."""
    L = ctypes.CDLL(path)
    L.or_assemble.restype = ctypes.c_int
    L.or_assemble.argtypes = [ctypes.POINTER(_Mesh), ctypes.POINTER(_Cfg),
                              ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                              ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.POINTER(_Res)]
    L.or_free.argtypes = [ctypes.POINTER(_Res)]
    L.or_region.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.POINTER(_Cfg),
                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                            ctypes.c_void_p]
    L.or_inner.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.POINTER(_Cfg),
                           ctypes.c_void_p, ctypes.c_void_p]
    L.or_rule_table.argtypes = [ctypes.c_int32, ctypes.c_void_p]
    L.or_gauss_legendre.argtypes = [ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
    L.or_record_hash.restype = ctypes.c_uint64
    L.or_record_hash.argtypes = [ctypes.c_int32] * 6
    L.or_hmax.restype = ctypes.c_double
    L.or_hmax.argtypes = [ctypes.POINTER(_Mesh)]
    return L


def _ptr(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


class _Keep:
    """Holds numpy buffers alive while ctypes structs point into them."""

    def __init__(self):
        self.bufs = []

    def arr(self, a, dtype):
        a = np.ascontiguousarray(a, dtype=dtype)
        self.bufs.append(a)
        return a


def _mesh_struct(mesh, keep):
    vx = keep.arr(mesh.vx, np.float64)
    vy = keep.arr(mesh.vy, np.float64)
    tri = keep.arr(np.asarray(mesh.tri).reshape(-1), np.int32)
    return _Mesh(vx.shape[0], tri.shape[0] // 3, _ptr(vx, ctypes.c_double), _ptr(vy, ctypes.c_double),
                 _ptr(tri, ctypes.c_int32))


def make_cfg(keep, delta, ball, outer="dunavant7", inner="dunavant7", kernel="const", kernel_c=1.0,
             ngon_off=None, cap_m=2, duffy_n=4, cap_printed=0, shifted=0):
    off = keep.arr(np.zeros((1, 2)) if ngon_off is None else ngon_off, np.float64)
    n = 0 if ngon_off is None else off.shape[0]
    return _Cfg(float(delta), float(kernel_c), KERNEL[kernel], BALL[ball], n, int(cap_m),
                _ptr(off, ctypes.c_double), RULE[outer], RULE[inner], int(duffy_n), int(cap_printed),
                int(shifted))


def cfg_of(problem, keep, **over):
    kw = dict(delta=problem.delta, ball=problem.ball, outer=problem.outer, inner=problem.inner,
              kernel=problem.kernel, kernel_c=problem.kernel_c, ngon_off=problem.ngon_off,
              cap_m=problem.cap_m)
    kw.update(over)
    return make_cfg(keep, **kw)


def assemble(mesh, cfg_kw: dict, a_list=None, row_mask=None, want_rec=False, want_hash=False,
             nthreads=0):
    """Assemble D by brute force over element pairs.  Returns a dict with the COO
    entries (row, col, val sorted by row then col), pair/qp-pair/interaction counts
    and optionally interaction records and per-outer-triangle hashes."""
    L = lib()
    keep = _Keep()
    m = _mesh_struct(mesh, keep)
    c = make_cfg(keep, **cfg_kw)
    al = None if a_list is None else keep.arr(a_list, np.int32)
    rm = None if row_mask is None else keep.arr(row_mask, np.uint8)
    r = _Res()
    rc = L.or_assemble(ctypes.byref(m), ctypes.byref(c),
                       None if al is None else al.ctypes.data, 0 if al is None else al.shape[0],
                       None if rm is None else rm.ctypes.data,
                       int(want_rec), int(want_hash), int(nthreads), ctypes.byref(r))
    if rc != 0:
        raise ValueError("oracle rejected the configuration")
    try:
        nnz = r.nnz
        out = dict(
            row=np.ctypeslib.as_array(r.row, (nnz,)).copy() if nnz else np.zeros(0, np.int32),
            col=np.ctypeslib.as_array(r.col, (nnz,)).copy() if nnz else np.zeros(0, np.int32),
            val=np.ctypeslib.as_array(r.val, (nnz,)).copy() if nnz else np.zeros(0),
            n_pairs=r.n_pairs, n_qp_pairs=r.n_qp_pairs, n_inter=r.n_inter, nv=m.nv)
        if want_rec:
            n = r.n_inter
            dt = np.dtype([("a", "<i4"), ("b", "<i4"), ("q", "i1"), ("kind", "i1"),
                           ("nverts", "i1"), ("ncaps", "i1")])
            buf = ctypes.string_at(r.rec, n * dt.itemsize) if n else b""
            out["rec"] = np.frombuffer(buf, dtype=dt).copy()
        if want_hash:
            K = m.nt
            out["hash_a"] = np.ctypeslib.as_array(r.hash_a, (K,)).copy()
            out["count_a"] = np.ctypeslib.as_array(r.count_a, (K,)).copy()
            out["qp_a"] = np.ctypeslib.as_array(r.qp_a, (K,)).copy()
    finally:
        L.or_free(ctypes.byref(r))
    return out


def to_csr(out, n=None):
    import scipy.sparse as sp
    n = out["nv"] if n is None else n
    return sp.csr_matrix((out["val"], (out["row"], out["col"])), shape=(n, n))


def region(tri_xy, x, cfg_kw):
    """Region R(x, T_b): (kind, polygon [n,2], caps [c,3] = (cx, cy, area))."""
    L = lib()
    keep = _Keep()
    c = make_cfg(keep, **cfg_kw)
    t = keep.arr(tri_xy, np.float64).reshape(-1)
    kind = np.zeros(1, np.int32)
    nv = np.zeros(1, np.int32)
    nc = np.zeros(1, np.int32)
    poly = np.zeros(2 * 128)
    caps = np.zeros(3 * 16)
    rc = L.or_region(t.ctypes.data, float(x[0]), float(x[1]), ctypes.byref(c), kind.ctypes.data,
                     nv.ctypes.data, poly.ctypes.data, nc.ctypes.data, caps.ctypes.data)
    if rc != 0:
        raise ValueError("oracle rejected the configuration")
    return int(kind[0]), poly[:2 * nv[0]].reshape(-1, 2).copy(), caps[:3 * nc[0]].reshape(-1, 3).copy()


def inner(tri_xy, x, cfg_kw):
    """Inner sums of R(x, T_b): s0, s1[3], S2[3,3] and the qp count."""
    L = lib()
    keep = _Keep()
    c = make_cfg(keep, **cfg_kw)
    t = keep.arr(tri_xy, np.float64).reshape(-1)
    out = np.zeros(13)
    nqp = np.zeros(1, np.int64)
    rc = L.or_inner(t.ctypes.data, float(x[0]), float(x[1]), ctypes.byref(c), out.ctypes.data, nqp.ctypes.data)
    if rc != 0:
        raise ValueError("oracle rejected the configuration")
    return out[0], out[1:4].copy(), out[4:13].reshape(3, 3).copy(), int(nqp[0])


def rule_table(name):
    L = lib()
    out = np.zeros((16, 4))
    n = L.or_rule_table(RULE[name], out.ctypes.data)
    return out[:n].copy()


def gauss_legendre(n):
    L = lib()
    x = np.zeros(n)
    w = np.zeros(n)
    L.or_gauss_legendre(n, x.ctypes.data, w.ctypes.data)
    return x, w


def record_hash(a, b, q, kind, nverts, ncaps):
    return int(lib().or_record_hash(int(a), int(b), int(q), int(kind), int(nverts), int(ncaps)))


def hmax(mesh):
    keep = _Keep()
    m = _mesh_struct(mesh, keep)
    return float(lib().or_hmax(ctypes.byref(m)))


# ---------------------------------------------------------------------------
# Load vector, right-hand side, direct solve, L2 error (numpy / scipy)
# ---------------------------------------------------------------------------

def load_vector(mesh, f_nodal):
    """G_j = int_{Omega} f phi_j over elements labelled Omega, f as a P1 interpolant:
    element mass matrix |T|/12 [[2,1,1],[1,2,1],[1,1,2]] (Eq. (lfunchj))."""
    tri = np.asarray(mesh.tri).reshape(-1, 3)
    x = mesh.vx[tri]
    y = mesh.vy[tri]
    area = 0.5 * np.abs((x[:, 1] - x[:, 0]) * (y[:, 2] - y[:, 0]) - (x[:, 2] - x[:, 0]) * (y[:, 1] - y[:, 0]))
    sel = np.asarray(mesh.elem_in_omega).astype(bool)
    fl = f_nodal[tri]
    G = np.zeros(mesh.vx.shape[0])
    for i in range(3):
        contrib = area * (2.0 * fl[:, i] + fl[:, (i + 1) % 3] + fl[:, (i + 2) % 3]) / 12.0
        np.add.at(G, tri[sel, i], contrib[sel])
    return G


def rhs(D, mesh, f_nodal, g_nodal):
    """F = G[Omega] - D[Omega, Omega_I] g[Omega_I]."""
    om = np.asarray(mesh.node_in_omega).astype(bool)
    G = load_vector(mesh, f_nodal)
    Dc = D.tocsr()
    return G[om] - Dc[om][:, ~om] @ g_nodal[~om]


def solve(D, mesh, f_nodal, g_nodal):
    """Direct solve of A U = F with A = D[Omega, Omega]; returns the full nodal vector."""
    import scipy.sparse.linalg as spla
    om = np.asarray(mesh.node_in_omega).astype(bool)
    A = D.tocsr()[om][:, om].tocsc()
    F = rhs(D, mesh, f_nodal, g_nodal)
    U = np.array(g_nodal, dtype=np.float64, copy=True)
    U[om] = spla.spsolve(A, F)
    return U


def l2_error_omega(mesh, U, u_exact, rule_name="dunavant16"):
    """|| u - u_h ||_{L2(Omega)} over elements labelled Omega."""
    tri = np.asarray(mesh.tri).reshape(-1, 3)
    sel = np.asarray(mesh.elem_in_omega).astype(bool)
    t = tri[sel]
    x = mesh.vx[t]
    y = mesh.vy[t]
    area = 0.5 * np.abs((x[:, 1] - x[:, 0]) * (y[:, 2] - y[:, 0]) - (x[:, 2] - x[:, 0]) * (y[:, 1] - y[:, 0]))
    R = rule_table(rule_name)
    err = 0.0
    for l0, l1, l2, w in R:
        px = l0 * x[:, 0] + l1 * x[:, 1] + l2 * x[:, 2]
        py = l0 * y[:, 0] + l1 * y[:, 1] + l2 * y[:, 2]
        uh = l0 * U[t[:, 0]] + l1 * U[t[:, 1]] + l2 * U[t[:, 2]]
        err += np.sum(w * area * (u_exact(px, py) - uh) ** 2)
    return float(np.sqrt(err))

"""FP64 CPU oracle (test infrastructure only).

Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
import this package.  It loads ``liboracle.so`` (plain C, single threaded,
built from ``oracle.c`` by ``build()``) and wraps it with numpy arrays.  It never
imports the CUDA package and shares no code with it.

Every function follows arXiv 2602.12365: Eq. 2 (discretised energy), Eq. 1
(residual as the gradient), Eq. 3 (tangent action as the JVP of the
residual), Algorithm 1 (gather / gradient / density / integrate / accumulate),
and the Dirichlet condensation of Sec. 6.1.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc -O2, no fast-math)."""
    src = os.path.join(_HERE, "oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < max(
            os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", _SO, src, "-lm"])
    return _SO


class NewtonOpts(C.Structure):
    _fields_ = [("newton_rtol", C.c_double), ("newton_max", C.c_int), ("eta_max", C.c_double),
                ("cg_max", C.c_int), ("predictor_rtol", C.c_double), ("armijo_c", C.c_double),
                ("ls_max", C.c_int), ("ls_eps", C.c_double), ("max_bisect", C.c_int)]


class NewtonStats(C.Structure):
    _fields_ = [("status", C.c_int), ("newton_iters", C.c_int), ("cg_iters", C.c_int),
                ("bisections", C.c_int), ("r0_norm", C.c_double), ("r_norm", C.c_double),
                ("ls_halvings", C.c_int)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_SO)
        P = C.c_void_p
        i64, i32, dbl = C.c_int64, C.c_int, C.c_double
        L.ora_nh_psi.restype = dbl
        L.ora_nh_psi.argtypes = [i32, P, dbl, dbl]
        L.ora_nh_P.argtypes = [i32, P, dbl, dbl, P]
        L.ora_nh_dP.argtypes = [i32, P, P, dbl, dbl, P]
        L.ora_geometry.restype = dbl
        L.ora_geometry.argtypes = [i32, P, i32, P, P]
        mesh = [i32, i64, i64, P, P, P, P]
        L.ora_energy.restype = dbl
        L.ora_energy.argtypes = mesh + [P, P, P, P]
        L.ora_residual.argtypes = mesh + [P, P, i32, P, P]
        L.ora_hvp.argtypes = mesh + [P, P, P, i32, i32, P, P]
        L.ora_block_diag.argtypes = mesh + [P, P, P, P]
        L.ora_param_vjp.argtypes = mesh + [P, P, P, P, P]
        L.ora_default_opts.argtypes = [P]
        L.ora_load_step.restype = i32
        L.ora_load_step.argtypes = mesh + [P, P, dbl, dbl, P, P, P]
        L.ora_mlp_forward.argtypes = [i32] * 5 + [P] * 8
        L.ora_mlp_backward.argtypes = [i32] * 5 + [P] * 15
        L.ora_node_graph.restype = i64
        L.ora_node_graph.argtypes = [i64, i64, i32, P, P, P, i64]
        L.ora_lp_features.argtypes = [i32, i64, i64, P, P, P, P, P, P]
        L.ora_lp_blocks.restype = i32
        L.ora_lp_blocks.argtypes = [i64, P, P, P, P]
        L.ora_lp_blocks_backward.argtypes = [i64, P, P, P, P, P]
        L.ora_ncm_set.restype = i32
        L.ora_ncm_set.argtypes = [i32, P]
        L.ora_ncm_eval.argtypes = [dbl, dbl, P, P, P]
        L.ora_law_psi.restype = dbl
        L.ora_law_psi.argtypes = [i32, P, dbl, dbl]
        L.ora_law_P.argtypes = [i32, P, dbl, dbl, P]
        L.ora_law_dP.argtypes = [i32, P, P, dbl, dbl, P]
        L.ora_dof_pattern.restype = i64
        L.ora_dof_pattern.argtypes = [i64, i32, i64, i32, P, P, P, i64]
        L.ora_distance2_colors.restype = i32
        L.ora_distance2_colors.argtypes = [i64, P, P, P]
        L.ora_sparse_values.restype = i32
        L.ora_sparse_values.argtypes = mesh + [P, P, i32, i32, P, P, P, P]
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class OracleMesh:
    """A mesh as the oracle sees it: FP64 coordinates, int32 connectivity,
    per-element moduli and the Dirichlet mask."""

    def __init__(self, elem_type, coords, conn, mu, lam, mask=None):
        self.etype = int(elem_type)
        self.X = _f64(coords)
        self.conn = np.ascontiguousarray(conn, dtype=np.int32)
        self.mu = _f64(mu)
        self.lam = _f64(lam)
        self.mask = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8).reshape(-1)
        self.dim = self.X.shape[1]
        self.nn = self.X.shape[0]
        self.ne = self.conn.shape[0]

    @classmethod
    def from_mesh(cls, m):
        return cls(m.elem_type, m.coords, m.conn, m.mu_e(), m.lam_e(), m.dirichlet)

    def _args(self):
        return (self.etype, self.nn, self.ne, _p(self.X), _p(self.conn), _p(self.mu), _p(self.lam))

    def energy(self, u, per_element=False):
        u = _f64(u).reshape(-1)
        st = C.c_int(0)
        asum = C.c_double(0)
        pe = np.zeros(self.ne) if per_element else None
        psi = lib().ora_energy(*self._args(), _p(u), _p(pe), C.byref(asum), C.byref(st))
        if per_element:
            return psi, pe, asum.value, st.value
        return psi

    def energy_status(self, u):
        u = _f64(u).reshape(-1)
        st = C.c_int(0)
        asum = C.c_double(0)
        psi = lib().ora_energy(*self._args(), _p(u), None, C.byref(asum), C.byref(st))
        return psi, asum.value, st.value

    def residual(self, u, mask_out=True, return_status=False):
        u = _f64(u).reshape(-1)
        r = np.zeros(self.nn * self.dim)
        st = C.c_int(0)
        lib().ora_residual(*self._args(), _p(u), _p(self.mask), int(mask_out), _p(r), C.byref(st))
        return (r, st.value) if return_status else r

    def hvp(self, u, v, mask_in=True, mask_out=True, return_status=False):
        u = _f64(u).reshape(-1)
        v = _f64(v).reshape(-1)
        y = np.zeros(self.nn * self.dim)
        st = C.c_int(0)
        lib().ora_hvp(*self._args(), _p(u), _p(v), _p(self.mask), int(mask_in), int(mask_out),
                      _p(y), C.byref(st))
        return (y, st.value) if return_status else y

    def sparse_K(self, u, mask_in=True, mask_out=True):
        """(ptr, idx, vals): K(u) on the DOF pattern, column j = K e_j (slow:
        one oracle HVP per DOF)."""
        ptr, idx = dof_pattern(self.nn, self.dim, self.conn)
        vals = np.zeros(idx.size)
        st = C.c_int(0)
        mk = self.mask if (mask_in or mask_out) else None
        rc = lib().ora_sparse_values(*self._args(), _p(_f64(u)), _p(mk), int(mask_in), int(mask_out),
                                     _p(ptr), _p(idx), _p(vals), C.byref(st))
        if rc != 0:
            raise RuntimeError("K e_j has entries outside the pattern")
        return ptr, idx, vals

    def block_diag(self, u):
        u = _f64(u).reshape(-1)
        D = np.zeros(self.nn * self.dim * self.dim)
        st = C.c_int(0)
        lib().ora_block_diag(*self._args(), _p(u), _p(self.mask), _p(D), C.byref(st))
        return D.reshape(self.nn, self.dim, self.dim)

    def param_vjp(self, u, a):
        u = _f64(u).reshape(-1)
        a = _f64(a).reshape(-1)
        gm = np.zeros(self.ne)
        gl = np.zeros(self.ne)
        st = C.c_int(0)
        lib().ora_param_vjp(*self._args(), _p(u), _p(a), _p(gm), _p(gl), C.byref(st))
        return gm, gl

    def load_step(self, ubar, s_prev, s, u, opts: NewtonOpts | None = None):
        """Advance u in place from load factor s_prev to s; returns stats."""
        assert u.dtype == np.float64 and u.flags.c_contiguous
        ub = _f64(ubar).reshape(-1)
        stats = NewtonStats()
        lib().ora_load_step(*self._args(), _p(self.mask), _p(ub), float(s_prev), float(s),
                            _p(u), None if opts is None else C.byref(opts), C.byref(stats))
        return stats


def default_opts() -> NewtonOpts:
    o = NewtonOpts()
    lib().ora_default_opts(C.byref(o))
    return o


def nh_psi(F, mu=1.0, lam=10.0):
    F = _f64(F)
    return lib().ora_nh_psi(F.shape[0], _p(F), mu, lam)


def nh_P(F, mu=1.0, lam=10.0):
    F = _f64(F)
    P = np.zeros_like(F)
    lib().ora_nh_P(F.shape[0], _p(F), mu, lam, _p(P))
    return P


def nh_dP(F, dF, mu=1.0, lam=10.0):
    F = _f64(F)
    dF = _f64(dF)
    dP = np.zeros_like(F)
    lib().ora_nh_dP(F.shape[0], _p(F), _p(dF), mu, lam, _p(dP))
    return dP


def geometry(etype, Xe, q):
    Xe = _f64(Xe)
    n_en, d = Xe.shape
    g = np.zeros((n_en, d))
    dJ = C.c_double(0)
    wdJ = lib().ora_geometry(etype, _p(Xe), q, _p(g), C.byref(dJ))
    return wdJ, dJ.value, g


def mlp_forward(x, W1, b1, W2, b2, W3, b3):
    x = _f64(x)
    n, d_in = x.shape
    h1, h2, d_out = W1.shape[0], W2.shape[0], W3.shape[0]
    y = np.zeros((n, d_out))
    Ws = [_f64(a) for a in (W1, b1, W2, b2, W3, b3)]
    lib().ora_mlp_forward(n, d_in, h1, h2, d_out, _p(x), *[_p(a) for a in Ws], _p(y))
    return y


def mlp_backward(x, W1, b1, W2, b2, W3, b3, gy):
    x = _f64(x)
    gy = _f64(gy)
    n, d_in = x.shape
    h1, h2, d_out = W1.shape[0], W2.shape[0], W3.shape[0]
    Ws = [_f64(a) for a in (W1, b1, W2, b2, W3, b3)]
    grads = [np.zeros_like(a) for a in Ws]
    gx = np.zeros_like(x)
    lib().ora_mlp_backward(n, d_in, h1, h2, d_out, _p(x), *[_p(a) for a in Ws], _p(gy),
                           *[_p(g) for g in grads], _p(gx))
    return grads, gx


# ----------------------------------------------------------------------------
# learned block preconditioner (3D): node graph, features, SPD blocks
# ----------------------------------------------------------------------------
LP_FEATURES = 36


def node_graph(n_nodes, conn):
    """CSR (ptr, idx) of the distinct nodes sharing an element with each node."""
    conn = np.ascontiguousarray(conn, dtype=np.int32)
    ne, n_en = conn.shape
    ptr = np.zeros(n_nodes + 1, np.int64)
    m = lib().ora_node_graph(n_nodes, ne, n_en, _p(conn), _p(ptr), None, 0)
    idx = np.zeros(max(m, 1), np.int32)
    lib().ora_node_graph(n_nodes, ne, n_en, _p(conn), _p(ptr), _p(idx), m)
    return ptr, idx[:m]


def lp_features(elem_type, conn, mu, lam, mask, D):
    """36 features per node from the diagonal blocks D [n_nodes, 3, 3]."""
    conn = np.ascontiguousarray(conn, dtype=np.int32)
    D = _f64(D).reshape(-1, 9)
    nn = D.shape[0]
    mk = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8).reshape(-1)
    F = np.zeros((nn, LP_FEATURES))
    lib().ora_lp_features(int(elem_type), nn, conn.shape[0], _p(conn), _p(_f64(mu)), _p(_f64(lam)),
                          None if mk is None else _p(mk), _p(D), _p(F))
    return F


def lp_blocks(D, mask, o):
    """M_i = F A A^T F^T / s_i (see oracle.c); returns (M [n, 3, 3], ok)."""
    D = _f64(D).reshape(-1, 9)
    o = _f64(o).reshape(-1, 6)
    mk = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8).reshape(-1)
    M = np.zeros((D.shape[0], 9))
    ok = lib().ora_lp_blocks(D.shape[0], _p(D), None if mk is None else _p(mk), _p(o), _p(M))
    return M.reshape(-1, 3, 3), bool(ok)


def lp_blocks_backward(D, mask, o, gM):
    D = _f64(D).reshape(-1, 9)
    o = _f64(o).reshape(-1, 6)
    gM = _f64(gM).reshape(-1, 9)
    mk = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8).reshape(-1)
    go = np.zeros((D.shape[0], 6))
    lib().ora_lp_blocks_backward(D.shape[0], _p(D), None if mk is None else _p(mk), _p(o), _p(gM), _p(go))
    return go


# ----------------------------------------------------------------------------
# sparse K by colouring (Sec. 2.2, Algorithm 2; App. A, B)
# ----------------------------------------------------------------------------
def dof_pattern(n_nodes, dim, conn):
    """CSR (ptr, idx) of the DOF pattern of K: entry (i, j) when the nodes of
    DOFs i and j share an element."""
    conn = np.ascontiguousarray(conn, dtype=np.int32)
    ne, n_en = conn.shape
    ptr = np.zeros(n_nodes * dim + 1, np.int64)
    m = lib().ora_dof_pattern(n_nodes, dim, ne, n_en, _p(conn), _p(ptr), None, 0)
    idx = np.zeros(max(m, 1), np.int32)
    lib().ora_dof_pattern(n_nodes, dim, ne, n_en, _p(conn), _p(ptr), _p(idx), m)
    return ptr, idx[:m]


def distance2_colors(ptr, idx):
    """Greedy distance-2 column colouring in ascending column order:
    (colors [n], n_colors)."""
    ptr = np.ascontiguousarray(ptr, dtype=np.int64)
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    n = ptr.size - 1
    col = np.zeros(max(n, 1), np.int32)
    nc = lib().ora_distance2_colors(n, _p(ptr), _p(idx), _p(col))
    return col[:n], int(nc)


# ----------------------------------------------------------------------------
# neural constitutive model (process-wide switch of the oracle's law)
# ----------------------------------------------------------------------------
class ncm:
    """Context manager: the oracle's element loops use psi = [NN(I1, J) -
    NN(3, 1)] + psi_NH inside the block (params as ora_ncm_set)."""

    def __init__(self, H, params):
        self.H = int(H)
        self.params = _f64(params)
        assert self.params.size == self.H * self.H + 5 * self.H + 1

    def __enter__(self):
        lib().ora_ncm_set(self.H, _p(self.params))
        return self

    def __exit__(self, *a):
        lib().ora_ncm_set(0, None)


def ncm_eval(I1, J):
    """(NN, gradient [2], Hessian [2, 2]) at (I1, J); needs an active ncm."""
    y = C.c_double(0.0)
    g = np.zeros(2)
    h = np.zeros(4)
    lib().ora_ncm_eval(float(I1), float(J), C.byref(y), _p(g), _p(h))
    return y.value, g, h.reshape(2, 2)


def law_psi(F, mu=1.0, lam=10.0):
    F = _f64(F)
    return lib().ora_law_psi(F.shape[0], _p(F), mu, lam)


def law_P(F, mu=1.0, lam=10.0):
    F = _f64(F)
    P = np.zeros_like(F)
    lib().ora_law_P(F.shape[0], _p(F), mu, lam, _p(P))
    return P


def law_dP(F, dF, mu=1.0, lam=10.0):
    F, dF = _f64(F), _f64(dF)
    dP = np.zeros_like(F)
    lib().ora_law_dP(F.shape[0], _p(F), _p(dF), mu, lam, _p(dP))
    return dP

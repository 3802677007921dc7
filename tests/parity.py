"""Per-node parity helpers (test infrastructure, shared by the GPU tests).

A whole-vector relative 2-norm can hide one bad node among many good ones.
These helpers bound the error at EACH node against the size of what was added
there: s_i = sum over the elements e touching node i of ||x_e,i||, the 2-norm
of element e's contribution to node i.  A summation of those contributions
in any order (the library adds them through its rounds and partial slots,
the oracle element by element) can differ from the exact sum by a few
roundings of that magnitude, so |x_gpu,i - x_oracle,i| <= tol * s_i is the
per-node form of the relative bars (1e-12 in FP64, 1e-5 in FP32).

The element contributions come from the oracle itself, evaluated on an
"exploded" copy of the elements: each element gets private copies of its
nodes, so the oracle's nodal result on that copy is exactly the list of
element contributions (Eq. 2 / Algorithm 1 element by element, nothing
summed across elements).
"""
from __future__ import annotations

import numpy as np

import oracle


def exploded(om: oracle.OracleMesh, els=None):
    """(mesh with private nodes per element, the element's global node ids)."""
    conn = om.conn if els is None else om.conn[els]
    ne, n_en = conn.shape
    mu = om.mu if els is None else om.mu[els]
    lam = om.lam if els is None else om.lam[els]
    ex = oracle.OracleMesh(om.etype, om.X[conn.reshape(-1)], np.arange(ne * n_en, dtype=np.int32).reshape(ne, n_en),
                           mu, lam, None)
    return ex, conn


def element_contributions(om: oracle.OracleMesh, u, v=None, els=None):
    """Per-element nodal contributions [n_el, n_en, dim] of the residual at u
    (v is None) or of the HVP at u along v, unmasked, and the node ids."""
    d = om.dim
    ex, conn = exploded(om, els)
    flat = conn.reshape(-1)
    ue = np.asarray(u, dtype=np.float64).reshape(-1, d)[flat].ravel()
    if v is None:
        c = ex.residual(ue, mask_out=False)
    else:
        ve = np.asarray(v, dtype=np.float64).reshape(-1, d)[flat].ravel()
        c = ex.hvp(ue, ve, mask_in=False, mask_out=False)
    return c.reshape(conn.shape[0], conn.shape[1], d), conn


def node_scale(n_nodes, conn, contrib):
    """s_i = sum over incident elements of ||x_e,i||_2."""
    d = contrib.shape[-1]
    s = np.zeros(n_nodes)
    np.add.at(s, conn.reshape(-1), np.linalg.norm(contrib.reshape(-1, d), axis=1))
    return s


def per_node_excess(x, x_ref, scale, tol, nodes=None):
    """Largest |x_i - x_ref,i| / (tol s_i) over the nodes (<= 1 passes); a node
    with s_i = 0 (no element) must match exactly.  x, x_ref: [n, dim]."""
    err = np.linalg.norm(np.asarray(x, np.float64) - np.asarray(x_ref, np.float64), axis=1)
    s = scale if nodes is None else scale[nodes]
    zero = s == 0
    if np.any(err[zero] != 0):
        return np.inf
    if np.all(zero):
        return 0.0
    return float(np.max(err[~zero] / (tol * s[~zero])))

"""Python face of the C ABI: a mesh handle and its element operators.

PyTorch supplies device memory and the current CUDA stream; each method only
marshals pointers and sizes into one C call.  Vectors are flat
``[n_nodes * dim]`` CUDA tensors (float64 for FEM_F64 calls, float32 for
FEM_F32 calls), node-major and interleaved.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib as L

# CUDA kernels each C-ABI call launches (tile kernel, plus the finalize kernel
# that sums the tile-shared nodes where there is one)
KERNELS_PER_CALL = {"energy": 1, "residual": 2, "hvp": 2, "block_diag": 2, "param_vjp": 1}


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.float64:
        return L.FEM_F64
    if t.dtype == torch.float32:
        return L.FEM_F32
    raise TypeError(f"unsupported dtype {t.dtype}")


def make_desc(elem_type, coords, conn, mu=None, lam=None, mu0=1.0, lam0=10.0, dirichlet=None,
              precision="mixed", tile_elems=0):
    """Build a MeshDesc plus the host arrays it points to (kept alive)."""
    keep = {
        "coords": np.ascontiguousarray(coords, dtype=np.float64),
        "conn": np.ascontiguousarray(conn, dtype=np.int32),
    }
    if mu is not None:
        keep["mu"] = np.ascontiguousarray(mu, dtype=np.float64)
        keep["lam"] = np.ascontiguousarray(lam, dtype=np.float64)
    if dirichlet is not None:
        keep["dir"] = np.ascontiguousarray(dirichlet, dtype=np.uint8)
    d = L.MeshDesc()
    d.elem_type = int(elem_type)
    d.precision = L.FEM_PREC_MIXED if precision == "mixed" else L.FEM_PREC_FP64
    d.n_nodes = keep["coords"].shape[0]
    d.n_elems = keep["conn"].shape[0]
    d.coords = keep["coords"].ctypes.data
    d.conn = keep["conn"].ctypes.data
    d.mu = keep["mu"].ctypes.data if "mu" in keep else None
    d.lam = keep["lam"].ctypes.data if "lam" in keep else None
    d.mu0 = float(mu0)
    d.lambda0 = float(lam0)
    d.dirichlet = keep["dir"].ctypes.data if "dir" in keep else None
    d.tile_elems = int(tile_elems)
    return d, keep


def plan_partition(elem_type, coords, conn, tile_elems=0):
    """Host-only partition (no GPU): per element tile, round (colour), lane and
    node ids in the vertex order the kernels use."""
    d, keep = make_desc(elem_type, coords, conn, tile_elems=tile_elems)
    ne = d.n_elems
    tile = np.zeros(ne, np.int32)
    rnd = np.zeros(ne, np.int64)
    lane = np.zeros(ne, np.int32)
    nodes = np.zeros(keep["conn"].shape, np.int32)
    info = L.MeshInfo()
    L.check(L.lib().fem_plan_partition(C.byref(d), tile.ctypes.data, rnd.ctypes.data,
                                       lane.ctypes.data, nodes.ctypes.data, C.byref(info)))
    return tile, rnd, lane, nodes, info.as_dict()


def sparse_pattern_host(elem_type, coords, conn):
    """Host-only DOF pattern of K and its greedy distance-2 column colouring
    (no GPU): (row_ptr int64, col_idx int32, colors int32, n_colors)."""
    d, keep = make_desc(elem_type, coords, conn)
    nnz, nc = C.c_int64(0), C.c_int32(0)
    L.check(L.lib().fem_sparse_pattern_desc(C.byref(d), C.byref(nnz), C.byref(nc), None, None, None))
    n_dofs = d.n_nodes * (2 if int(elem_type) == 0 else 3)
    rp = np.zeros(n_dofs + 1, np.int64)
    ci = np.zeros(max(nnz.value, 1), np.int32)
    co = np.zeros(n_dofs, np.int32)
    L.check(L.lib().fem_sparse_pattern_desc(C.byref(d), None, None, rp.ctypes.data_as(C.c_void_p),
                                            ci.ctypes.data_as(C.c_void_p), co.ctypes.data_as(C.c_void_p)))
    return rp, ci[:nnz.value], co, nc.value


class Mesh:
    """A mesh uploaded to the GPU (owns the C handle)."""

    def __init__(self, elem_type, coords, conn, mu=None, lam=None, mu0=1.0, lam0=10.0,
                 dirichlet=None, precision="mixed", tile_elems=0, stream=None):
        d, keep = make_desc(elem_type, coords, conn, mu, lam, mu0, lam0, dirichlet, precision,
                            tile_elems)
        h = C.c_void_p()
        L.check(L.lib().fem_mesh_create(C.byref(d), C.byref(h), _stream(stream)))
        self._h = h
        self.elem_type = int(elem_type)
        self.dim = 2 if elem_type == 0 else 3
        self.n_nodes = int(d.n_nodes)
        self.n_el = int(d.n_elems)
        self.precision = precision
        self.mask = None
        if dirichlet is not None:
            self.mask = torch.as_tensor(keep["dir"].reshape(-1).astype(bool)).cuda()

    @classmethod
    def from_fixture(cls, m, precision="mixed", tile_elems=0):
        return cls(m.elem_type, m.coords, m.conn, m.mu, m.lam, m.mu0, m.lam0, m.dirichlet,
                   precision, tile_elems)

    def close(self):
        if getattr(self, "_h", None):
            L.lib().fem_mesh_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def dirichlet_mask(self, device=None) -> torch.Tensor:
        """Boolean per-DOF mask of the prescribed components (all False
        without Dirichlet data)."""
        if self.mask is None:
            return torch.zeros(self.n_nodes * self.dim, dtype=torch.bool, device=device or "cuda")
        return self.mask if device is None else self.mask.to(device)

    @property
    def n_dofs(self):
        return self.n_nodes * self.dim

    def info(self) -> dict:
        i = L.MeshInfo()
        L.check(L.lib().fem_mesh_get_info(self._h, C.byref(i)))
        return i.as_dict()

    def _check_vec(self, *ts):
        for t in ts:
            if not (t.is_cuda and t.is_contiguous() and t.numel() == self.n_dofs):
                raise ValueError("vectors must be contiguous CUDA tensors of n_nodes*dim entries")

    # --- element operators -------------------------------------------------
    def energy(self, u, out=None, stream=None):
        """Device double[4]: Psi, roundoff scale S, #(J <= 0), 0."""
        self._check_vec(u)
        out = out if out is not None else torch.empty(4, dtype=torch.float64, device=u.device)
        L.check(L.lib().fem_energy(self._h, _dtype_code(u), _ptr(u), _ptr(out), _stream(stream)))
        return out

    def energy_static(self, u, out=None, stream=None):
        """energy() through fem_energy_static: reduction scratch in a fixed
        module-scope device array, no allocation; calls must not overlap."""
        self._check_vec(u)
        out = out if out is not None else torch.empty(4, dtype=torch.float64, device=u.device)
        L.check(L.lib().fem_energy_static(self._h, _dtype_code(u), _ptr(u), _ptr(out), _stream(stream)))
        return out

    def residual(self, u, mask_out=True, out=None, stream=None):
        self._check_vec(u)
        out = out if out is not None else torch.empty_like(u)
        L.check(L.lib().fem_residual(self._h, _dtype_code(u), _ptr(u), _ptr(out),
                                     L.FEM_MASK_OUT if mask_out else 0, _stream(stream)))
        return out

    def hvp(self, u, v, mask_in=True, mask_out=True, out=None, vkv=None, stream=None):
        self._check_vec(u, v)
        if u.dtype != v.dtype:
            raise TypeError("u and v must have the same dtype")
        out = out if out is not None else torch.empty_like(u)
        flags = (L.FEM_MASK_IN if mask_in else 0) | (L.FEM_MASK_OUT if mask_out else 0)
        L.check(L.lib().fem_hvp(self._h, _dtype_code(u), _ptr(u), _ptr(v), _ptr(out), flags,
                                _ptr(vkv), _stream(stream)))
        return out

    def block_diag(self, u, out=None, stream=None):
        self._check_vec(u)
        out = out if out is not None else torch.empty(self.n_nodes * self.dim * self.dim,
                                                      dtype=u.dtype, device=u.device)
        L.check(L.lib().fem_block_diag(self._h, _dtype_code(u), _ptr(u), _ptr(out), _stream(stream)))
        return out

    # --- neural constitutive model -------------------------------------------
    def set_ncm(self, hidden: int, params=None):
        """psi = [NN(I1, J) - NN(3, 1)] + psi_NH for every operator of this
        mesh (fem_mesh_set_ncm); hidden = 0 restores the Neo-Hookean law."""
        if hidden == 0:
            L.check(L.lib().fem_mesh_set_ncm(self._h, 0, None))
            return
        p = np.ascontiguousarray(params, dtype=np.float64)
        if p.size != hidden * hidden + 5 * hidden + 1:
            raise ValueError("params must hold H*H + 5H + 1 values")
        L.check(L.lib().fem_mesh_set_ncm(self._h, int(hidden), p.ctypes.data_as(C.c_void_p)))

    # --- ablation: element-per-thread scatter with float atomics ---------------
    def residual_atomic(self, u, mask_out=True, out=None, stream=None):
        """fem_residual_atomic: the residual by atomic scatter-add (run-to-run
        bit differences possible)."""
        self._check_vec(u)
        out = out if out is not None else torch.empty_like(u)
        L.check(L.lib().fem_residual_atomic(self._h, _dtype_code(u), _ptr(u), _ptr(out),
                                            L.FEM_MASK_OUT if mask_out else 0, _stream(stream)))
        return out

    def hvp_atomic(self, u, v, mask_in=True, mask_out=True, out=None, stream=None):
        """fem_hvp_atomic: the HVP by atomic scatter-add."""
        self._check_vec(u, v)
        out = out if out is not None else torch.empty_like(u)
        flags = (L.FEM_MASK_IN if mask_in else 0) | (L.FEM_MASK_OUT if mask_out else 0)
        L.check(L.lib().fem_hvp_atomic(self._h, _dtype_code(u), _ptr(u), _ptr(v), _ptr(out), flags,
                                       _stream(stream)))
        return out

    def sparse_assemble_atomic(self, u, mask_in=True, mask_out=True, out=None, stream=None):
        """fem_sparse_assemble_atomic: K by element stiffness and atomic
        scatter-add into the CSR values (run-to-run bit differences possible)."""
        self._check_vec(u)
        nnz, _ = self.sparse_info()
        out = out if out is not None else torch.empty(nnz, dtype=u.dtype, device=u.device)
        flags = (L.FEM_MASK_IN if mask_in else 0) | (L.FEM_MASK_OUT if mask_out else 0)
        L.check(L.lib().fem_sparse_assemble_atomic(self._h, _dtype_code(u), _ptr(u), flags, _ptr(out),
                                                   _stream(stream)))
        return out

    # --- sparse K by colouring (Algorithm 2) ----------------------------------
    def sparse_info(self):
        """(nnz, n_colors) of K's DOF pattern and its distance-2 colouring
        (built on the host by the first call)."""
        nnz, nc = C.c_int64(0), C.c_int32(0)
        L.check(L.lib().fem_sparse_info(self._h, C.byref(nnz), C.byref(nc)))
        return nnz.value, nc.value

    def sparse_pattern(self):
        """Host numpy (row_ptr int64, col_idx int32, colors int32)."""
        nnz, _ = self.sparse_info()
        rp = np.zeros(self.n_dofs + 1, np.int64)
        ci = np.zeros(max(nnz, 1), np.int32)
        co = np.zeros(self.n_dofs, np.int32)
        L.check(L.lib().fem_sparse_pattern(self._h, rp.ctypes.data_as(C.c_void_p), ci.ctypes.data_as(C.c_void_p),
                                           co.ctypes.data_as(C.c_void_p)))
        return rp, ci[:nnz], co

    def sparse_assemble(self, u, mask_in=True, mask_out=True, out=None, stream=None):
        """CSR values of Mo K(u) Mi on the pattern (device, u's dtype): one
        HVP per colour, then the decompression of Algorithm 2."""
        self._check_vec(u)
        nnz, _ = self.sparse_info()
        out = out if out is not None else torch.empty(nnz, dtype=u.dtype, device=u.device)
        if not (out.is_cuda and out.is_contiguous() and out.numel() == nnz and out.dtype == u.dtype):
            raise ValueError("out must be a contiguous CUDA tensor of nnz entries in u's dtype")
        flags = (L.FEM_MASK_IN if mask_in else 0) | (L.FEM_MASK_OUT if mask_out else 0)
        L.check(L.lib().fem_sparse_assemble(self._h, _dtype_code(u), _ptr(u), flags, _ptr(out), _stream(stream)))
        return out

    def sparse_spmv(self, values, x, out=None, stream=None):
        """y = K x with the pattern and `values` (device, x's dtype)."""
        self._check_vec(x)
        if values.dtype != x.dtype or not (values.is_cuda and values.is_contiguous()):
            raise TypeError("values must be a contiguous CUDA tensor of x's dtype")
        out = out if out is not None else torch.empty_like(x)
        L.check(L.lib().fem_sparse_spmv(self._h, _dtype_code(x), _ptr(values), _ptr(x), _ptr(out), _stream(stream)))
        return out

    def param_vjp(self, u, a, stream=None):
        self._check_vec(u, a)
        gm = torch.empty(self.n_el, dtype=torch.float64, device=u.device)
        gl = torch.empty(self.n_el, dtype=torch.float64, device=u.device)
        L.check(L.lib().fem_param_vjp(self._h, _dtype_code(u), _ptr(u), _ptr(a), _ptr(gm), _ptr(gl),
                                      _stream(stream)))
        return gm, gl

    def newton_step(self, u, ubar, s_prev, s, cg_dtype=torch.float64, check=True, stream=None,
                    **opts):
        """One Newton-CG load step from s_prev to s (fem_newton_step); u (FP64,
        on the device) is updated in place.  ``cg_dtype`` float32 runs the PCG
        in FP32 with FP64 dots; ``learned=`` a LearnedPreconditioner selects
        the learned block preconditioner; other keyword ``opts`` override
        fem_newton_opts fields.  Returns the step statistics as a dict; with ``check`` a
        failed step raises FemError."""
        if u.dtype != torch.float64 or ubar.dtype != torch.float64:
            raise TypeError("u and ubar must be float64 (the master state is FP64)")
        self._check_vec(u, ubar)
        o = L.NewtonOpts()
        L.check(L.lib().fem_newton_default_opts(C.byref(o)))
        o.cg_dtype = L.FEM_F64 if cg_dtype == torch.float64 else L.FEM_F32
        learned = opts.pop("learned", None)
        if learned is not None:  # a LearnedPreconditioner
            o.precond = L.FEM_PC_LEARNED
            o.learned = learned.handle.value
        for k, v in opts.items():
            if not hasattr(o, k):
                raise TypeError(f"unknown option {k}")
            setattr(o, k, v)
        st = L.NewtonStats()
        rc = L.lib().fem_newton_step(self._h, _ptr(u), _ptr(ubar), float(s_prev), float(s),
                                     C.byref(o), C.byref(st), _stream(stream))
        if check:
            L.check(rc)
        return st.as_dict()

    def tangent_solve(self, u, b, rtol=1e-8, cg_dtype=torch.float64, cg_max=0, stream=None, check=True):
        """x with M K(u) M x = M b (block-Jacobi PCG, fem_tangent_solve);
        returns (x, iterations), or (x, iterations, status) with
        ``check=False`` (x is the last iterate when the cap is reached)."""
        if u.dtype != torch.float64 or b.dtype != torch.float64:
            raise TypeError("u and b must be float64")
        self._check_vec(u, b)
        x = torch.empty_like(u)
        it = C.c_int64(0)
        rc = L.lib().fem_tangent_solve(self._h, L.FEM_F64 if cg_dtype == torch.float64 else L.FEM_F32,
                                       _ptr(u), _ptr(b), _ptr(x), float(rtol), int(cg_max),
                                       C.byref(it), _stream(stream))
        if check:
            L.check(rc)
            return x, it.value
        return x, it.value, rc

    def set_moduli(self, mu, lam, stream=None):
        """Replace the per-element moduli (host arrays, element order)."""
        mu = np.ascontiguousarray(mu, dtype=np.float64).reshape(-1)
        lam = np.ascontiguousarray(lam, dtype=np.float64).reshape(-1)
        if mu.size != self.n_el or lam.size != self.n_el:
            raise ValueError("mu and lam need one value per element")
        L.check(L.lib().fem_mesh_set_moduli(self._h, mu.ctypes.data_as(C.c_void_p), lam.ctypes.data_as(C.c_void_p),
                                            _stream(stream)))

    def compliance_gradient(self, u, ratio=10.0, rtol=1e-10, cg_dtype=torch.float64, vjp_dtype=torch.float64,
                            stream=None):
        """(c, dc/dmu [n_elems] FP64, adjoint PCG iterations) at the converged
        FP64 state u, all of it in the library (fem_compliance_gradient)."""
        if u.dtype != torch.float64:
            raise TypeError("u must be float64 (the master state is FP64)")
        self._check_vec(u)
        g = torch.empty(self.n_el, dtype=torch.float64, device=u.device)
        c = torch.empty(1, dtype=torch.float64, device=u.device)
        it = C.c_int64(0)
        code = {torch.float64: L.FEM_F64, torch.float32: L.FEM_F32}
        L.check(L.lib().fem_compliance_gradient(self._h, _ptr(u), float(ratio), float(rtol), code[cg_dtype],
                                                code[vjp_dtype], _ptr(g), _ptr(c), C.byref(it), _stream(stream)))
        return c, g, it.value

    def sync_status(self, stream=None) -> int:
        f = C.c_int32(0)
        L.check(L.lib().fem_sync_status(self._h, _stream(stream), C.byref(f)))
        return f.value


def fp32_fma_rate(blocks, iters, out, stream=None):
    """Enqueue the FP32 FMA throughput kernel (fem_fp32_fma_rate) writing
    `out` (device float32 [blocks * 256]); returns its FLOP count."""
    if out.dtype != torch.float32 or not out.is_cuda or out.numel() < blocks * 256:
        raise ValueError("out must be a CUDA float32 tensor of at least blocks * 256 elements")
    fl = C.c_double(0.0)
    L.check(L.lib().fem_fp32_fma_rate(int(blocks), int(iters), _ptr(out), C.byref(fl), _stream(stream)))
    return fl.value

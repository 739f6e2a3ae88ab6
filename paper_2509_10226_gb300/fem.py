"""Thin PyTorch-facing wrapper over the tetmf C ABI.

Every computation runs in the CUDA library; this module only passes device
pointers (``tensor.data_ptr()``), sizes and the current CUDA stream.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import call

PREC = {"fp64": _lib.FEM_FP64, "fp32": _lib.FEM_FP32, "tf32": _lib.FEM_TF32, "bf16": _lib.FEM_BF16,
        "tf32x3": _lib.FEM_TF32X3}


def _vec_dtype(prec: str):
    return torch.float64 if prec == "fp64" else torch.float32


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class FemSpace:
    """A mesh + finite-element space + device plan (one fem_ctx).

    xyz [nv, 3] float64 and cells [nc, 4] int32 are host arrays in the user's
    numbering.  device = -1 builds a host-only plan (queries only).  modified_rule selects the
    cell rule exact to degree 2p - 2 (Sec. 3.3; faces keep the standard rule).  scatter = "colour"
    (CG) orders the cells by colour and adds without atomics in the FP64/FP32 apply (reproducible).
    cell_nodes [n_cells, 10, 3] makes the cells curved (second-order geometry, CG).
    """

    def __init__(self, xyz, cells, kind="cg", degree=1, dirichlet=False, reorder=True, penalty=None, device=0,
                 modified_rule=False, scatter="atomic", cell_nodes=None):
        xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        cells = np.ascontiguousarray(cells, dtype=np.int32)
        nodes = None if cell_nodes is None else np.ascontiguousarray(cell_nodes, dtype=np.float64)
        if nodes is not None and nodes.shape != (cells.shape[0], 10, 3):
            raise ValueError("cell_nodes must be [n_cells, 10, 3]")
        mesh = _lib.MeshDesc(xyz.shape[0], xyz.ctypes.data, cells.shape[0], cells.ctypes.data,
                             None if nodes is None else nodes.ctypes.data)
        space = _lib.SpaceDesc(_lib.FEM_CG if kind == "cg" else _lib.FEM_DG, int(degree), int(bool(dirichlet)),
                               _lib.FEM_REORDER_MORTON if reorder else _lib.FEM_REORDER_NONE,
                               float(penalty) if penalty else 0.0, int(device),
                               _lib.FEM_RULE_MODIFIED if modified_rule else _lib.FEM_RULE_STANDARD,
                               _lib.FEM_SCATTER_COLOUR if scatter == "colour" else _lib.FEM_SCATTER_ATOMIC)
        h = ctypes.c_void_p()
        call("fem_create", ctypes.byref(mesh), ctypes.byref(space), ctypes.byref(h))
        self._h = h
        self.kind, self.degree, self.device = kind, int(degree), int(device)
        self.n_dofs = self._q64("fem_num_dofs")
        self.n_cells = self._q64("fem_num_cells")
        self.dofs_per_cell = self._q32("fem_dofs_per_cell")
        self.n_qpoints = self._q32("fem_num_qpoints")
        a, b = ctypes.c_int64(), ctypes.c_int64()
        call("fem_num_faces", self._h, ctypes.byref(a), ctypes.byref(b))
        self.n_interior_faces, self.n_boundary_faces = a.value, b.value

    def _q64(self, name):
        v = ctypes.c_int64()
        call(name, self._h, ctypes.byref(v))
        return v.value

    def _q32(self, name):
        v = ctypes.c_int32()
        call(name, self._h, ctypes.byref(v))
        return v.value

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            _lib.lib().fem_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- numbering -----------------------------------------------------
    def cell_permutation(self):
        out = np.empty(self.n_cells, dtype=np.int32)
        call("fem_cell_permutation", self._h, out.ctypes.data)
        return out

    def dof_permutation(self):
        out = np.empty(self.n_dofs, dtype=np.int64)
        call("fem_dof_permutation", self._h, out.ctypes.data)
        return out

    def dof_keys(self):
        out = np.empty((self.n_dofs, self.degree), dtype=np.int32)
        call("fem_dof_keys", self._h, out.ctypes.data)
        return out

    def colour_starts(self):
        """First library cell of each colour and the end ([n_colours + 1]); empty in atomic mode."""
        n = ctypes.c_int32()
        call("fem_colours", self._h, ctypes.byref(n), None)
        out = np.empty(n.value + 1 if n.value else 0, dtype=np.int64)
        if n.value:
            call("fem_colours", self._h, ctypes.byref(n), out.ctypes.data)
        return out

    def dof_coordinates(self):
        """Node positions of the library DoFs, [N, 3] float64 (host)."""
        out = np.empty((self.n_dofs, 3), dtype=np.float64)
        call("fem_dof_coordinates", self._h, out.ctypes.data)
        return out

    def dirichlet_mask(self):
        out = np.empty(self.n_dofs, dtype=np.uint8)
        call("fem_dirichlet_mask", self._h, out.ctypes.data)
        return out.astype(bool)

    def device_status(self):
        """Device error word (0 = clean), reset after reading; synchronises the device."""
        v = ctypes.c_int32()
        call("fem_device_status", self._h, ctypes.byref(v))
        return v.value

    def selftest_wait(self, limit_s=0.05):
        """Run the bounded-wait diagnostics (waits that nothing completes give up after limit_s);
        returns the two waits' durations in seconds.  Sets bit 0 of the device status word."""
        w = (ctypes.c_int64 * 2)()
        call("fem_selftest_wait", self._h, int(limit_s * 1e9), w)
        return w[0] * 1e-9, w[1] * 1e-9

    # ---- hot calls -------------------------------------------------------
    def _check_vec(self, t, prec, name, n=None):
        n = self.n_dofs if n is None else n
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == _vec_dtype(prec) and t.is_contiguous()
                and t.numel() == n):
            raise ValueError(f"{name}: need a contiguous CUDA tensor of {n} {_vec_dtype(prec)} values")

    def _check_k(self, k, prec):
        if k is not None:
            self._check_vec(k, prec, "k", self.n_cells * self.n_qpoints)

    def apply(self, u, k=None, prec="fp64", out=None, stream=None):
        """y = A(k) u (library DoF order)."""
        self._check_vec(u, prec, "u")
        self._check_k(k, prec)
        y = torch.empty_like(u) if out is None else out
        call("fem_apply", self._h, PREC[prec], _ptr(u), _ptr(y), _ptr(k), _stream(stream))
        return y

    def apply_host(self, us, ys, prec="fp64"):
        """ys[b] = A us[b] for host (CPU) tensors us[b], ys[b] of n_dofs values (a stream of
        requests through the device; blocking).  Pinned tensors give the full link bandwidth; a
        tensor may appear several times in ys (its last vector wins)."""
        if len(us) != len(ys) or not us:
            raise ValueError("us and ys must be equally long, non-empty sequences")
        dt = _vec_dtype(prec)
        for t in list(us) + list(ys):
            if not (isinstance(t, torch.Tensor) and not t.is_cuda and t.dtype == dt and t.is_contiguous()
                    and t.numel() == self.n_dofs):
                raise ValueError("host vectors must be contiguous CPU tensors of n_dofs values of the precision's type")
        n = len(us)
        up = (ctypes.c_void_p * n)(*[t.data_ptr() for t in us])
        yp = (ctypes.c_void_p * n)(*[t.data_ptr() for t in ys])
        call("fem_apply_host", self._h, PREC[prec], n, up, yp)
        return ys

    def apply_vector(self, u, prec="fp64", out=None, stream=None):
        """y[c] = A u[c] for the components c of u [ncomp, N] (vector Laplacian)."""
        if not (isinstance(u, torch.Tensor) and u.is_cuda and u.dim() == 2 and u.shape[1] == self.n_dofs
                and u.dtype == _vec_dtype(prec) and u.is_contiguous()):
            raise ValueError("u must be a contiguous CUDA tensor [ncomp, n_dofs] of the precision's vector type")
        y = torch.empty_like(u) if out is None else out
        call("fem_apply_vector", self._h, PREC[prec], int(u.shape[0]), _ptr(u), _ptr(y), _stream(stream))
        return y

    def apply_adjoint(self, g, k=None, prec="fp64", out=None, stream=None):
        self._check_vec(g, prec, "g")
        self._check_k(k, prec)
        y = torch.empty_like(g) if out is None else out
        call("fem_apply_adjoint", self._h, PREC[prec], _ptr(g), _ptr(y), _ptr(k), _stream(stream))
        return y

    def coeff_grad(self, u, g, k=None, prec="fp64", stream=None):
        """(grad_u, dk) of L = <g, A(k) u>."""
        self._check_vec(u, prec, "u")
        self._check_vec(g, prec, "g")
        self._check_k(k, prec)
        gu = torch.empty_like(u)
        dk = torch.empty(self.n_cells, self.n_qpoints, dtype=u.dtype, device=u.device)
        call("fem_coeff_grad", self._h, PREC[prec], _ptr(u), _ptr(g), _ptr(k), _ptr(gu), _ptr(dk), _stream(stream))
        return gu, dk

    def diagonal(self, k=None, prec="fp64", stream=None):
        self._check_k(k, prec)
        d = torch.empty(self.n_dofs, dtype=_vec_dtype(prec), device=f"cuda:{self.device}")
        call("fem_diagonal", self._h, PREC[prec], _ptr(d), _ptr(k), _stream(stream))
        return d

    def rhs_const(self, f=1.0, stream=None):
        b = torch.empty(self.n_dofs, dtype=torch.float64, device=f"cuda:{self.device}")
        call("fem_rhs_const", self._h, ctypes.c_double(f), _ptr(b), _stream(stream))
        return b

    def csr_build(self):
        nnz = ctypes.c_int64()
        call("fem_csr_build", self._h, ctypes.byref(nnz))
        return nnz.value

    def csr_apply(self, u, prec="fp64", out=None, stream=None):
        self._check_vec(u, prec, "u")
        y = torch.empty_like(u) if out is None else out
        call("fem_csr_apply", self._h, PREC[prec], _ptr(u), _ptr(y), _stream(stream))
        return y

    def _smoother_work(self, prec):
        nb = ctypes.c_int64()
        call("fem_smoother_work_bytes", self._h, PREC[prec], ctypes.byref(nb))
        return torch.empty(nb.value, dtype=torch.uint8, device=f"cuda:{self.device}")

    def chebyshev(self, b, x, diag, degree=5, lam_max=None, ratio=15.0, prec="fp64", stream=None):
        """degree steps of Chebyshev-Jacobi smoothing of A x = b, x updated in place; lam_max bounds
        the spectrum of diag^-1 A (see lambda_max)."""
        for t, name in ((b, "b"), (x, "x"), (diag, "diag")):
            self._check_vec(t, prec, name)
        work = self._smoother_work(prec)
        call("fem_chebyshev", self._h, PREC[prec], _ptr(b), _ptr(x), _ptr(diag), int(degree), float(lam_max),
             float(ratio), _ptr(work), _stream(stream))
        return x

    def lambda_max(self, diag, v0, iterations=20, prec="fp64", stream=None):
        """Power-iteration estimate of the largest eigenvalue of diag^-1 A (blocking)."""
        self._check_vec(diag, prec, "diag")
        self._check_vec(v0, prec, "v0")
        work = self._smoother_work(prec)
        lam = ctypes.c_double()
        call("fem_lambda_max", self._h, PREC[prec], _ptr(diag), _ptr(v0), int(iterations), _ptr(work),
             ctypes.byref(lam), _stream(stream))
        return lam.value

    def solve(self, b, x0=None, mode="ir", inner_prec="fp32", rtol=1e-10, inner_rtol=1e-3, max_outer=50,
              max_inner=20000, stream=None, raise_on_notconv=True, no_alloc=False, smoother_degree=0,
              coarse_steps=0):
        """Solve A x = b (blocking).  Returns (x, stats dict).  mode: "pcg" (FP64 Jacobi-PCG), "ir"
        (FP64 refinement around FP32-vector Jacobi-PCG), "pmg" (the same refinement around flexible
        CG with a p-multigrid V-cycle).

        no_alloc=True calls fem_solve_noalloc: the same solver with its work space in
        the library's fixed device array instead of memory the context allocates (for
        callers whose device memory must not be allocated by the library; at most
        FEM_SOLVE_NOALLOC_MAX_DOFS unknowns, concurrent calls must be serialised)."""
        self._check_vec(b, "fp64", "b")
        x = torch.zeros_like(b) if x0 is None else x0.clone()
        modes = {"ir": _lib.FEM_SOLVE_IR_MIXED, "pcg": _lib.FEM_SOLVE_FP64_PCG, "pmg": _lib.FEM_SOLVE_IR_PMG}
        opts = _lib.SolveOpts(modes[mode], PREC[inner_prec], rtol, inner_rtol, max_outer, max_inner,
                              int(smoother_degree), int(coarse_steps))
        st = _lib.SolveStats()
        fn = _lib.lib().fem_solve_noalloc if no_alloc else _lib.lib().fem_solve
        status = fn(self._h, ctypes.byref(opts), _ptr(b), _ptr(x), ctypes.byref(st), _stream(stream))
        stats = {"outer": st.outer_iterations, "inner": st.inner_iterations, "rel_residual": st.rel_residual,
                 "seconds": st.seconds, "converged": status == _lib.FEM_OK}
        if status != _lib.FEM_OK and (status != _lib.FEM_ENOTCONV or raise_on_notconv):
            _lib.check(status, "fem_solve_noalloc" if no_alloc else "fem_solve")
        return x, stats


class Transfer:
    """Prolongation / restriction between two CG spaces of different degree on one mesh."""

    def __init__(self, fine: FemSpace, coarse: FemSpace):
        h = ctypes.c_void_p()
        call("fem_transfer_create", fine._h, coarse._h, ctypes.byref(h))
        self._h, self.fine, self.coarse = h, fine, coarse  # the spaces must outlive the transfer

    def close(self):
        if getattr(self, "_h", None):
            _lib.lib().fem_transfer_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass

    def prolongate(self, uc, prec="fp64", out=None, stream=None):
        self.coarse._check_vec(uc, prec, "u_coarse")
        uf = torch.empty(self.fine.n_dofs, dtype=uc.dtype, device=uc.device) if out is None else out
        call("fem_prolongate", self._h, PREC[prec], _ptr(uc), _ptr(uf), _stream(stream))
        return uf

    def restrict(self, rf, prec="fp64", out=None, stream=None):
        self.fine._check_vec(rf, prec, "r_fine")
        rc = torch.empty(self.coarse.n_dofs, dtype=rf.dtype, device=rf.device) if out is None else out
        call("fem_restrict", self._h, PREC[prec], _ptr(rf), _ptr(rc), _stream(stream))
        return rc


class FemApply(torch.autograd.Function):
    """y = A(k) u with a hand-written backward (fem_coeff_grad):
    dL/du = A(k)^T (dL/dy) and dL/dk_{e,q} = w_q |det J_e| (grad u . grad dL/dy)."""

    @staticmethod
    def forward(ctx, space: FemSpace, u, k, prec="fp64"):
        ctx.space, ctx.prec = space, prec
        ctx.save_for_backward(u, k)
        return space.apply(u.contiguous(), k=None if k is None else k.contiguous(), prec=prec)

    @staticmethod
    def backward(ctx, gy):
        u, k = ctx.saved_tensors
        gy = gy.contiguous()
        gu, dk = ctx.space.coeff_grad(u.contiguous(), gy, k=None if k is None else k.contiguous(), prec=ctx.prec)
        return None, gu, (dk.reshape(k.shape) if k is not None and ctx.needs_input_grad[2] else None), None


def fem_apply(space: FemSpace, u, k=None, prec="fp64"):
    return FemApply.apply(space, u, k, prec)


def fma_probe(kind: str, iters: int, sink, stream=None):
    """Launch the library's arithmetic-throughput probe (fem_fma_probe) on the current device:
    kind "fp64", "fp32" or "fp32x2"; sink is a device tensor of at least one float64.  Returns the
    floating-point operations launched; time the call with events on `stream`."""
    flops = ctypes.c_double()
    call("fem_fma_probe", {"fp64": 0, "fp32": 1, "fp32x2": 2}[kind], int(iters), _ptr(sink), ctypes.byref(flops),
         _stream(stream))
    return flops.value

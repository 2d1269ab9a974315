"""Python convenience layer over libdpp: torch tensors in, torch tensors out.

torch serves only as device memory and streams here. Every computation of the
solver path (assembly, preconditioner setup, Krylov solve, adjoint) runs in
libdpp's CUDA kernels, called through the ctypes binding.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B


def _dev(a, dtype, device) -> torch.Tensor:
    if isinstance(a, torch.Tensor):
        return a.to(device=device, dtype=dtype).contiguous()
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device=device)


def _stream(device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


class DPPSystem:
    """One assembled DPP system (problem handle) and optionally its preconditioner."""

    def __init__(self, coords, cells, bfacets, log_k1, log_k2, mu, beta, gamma_b, p01, p02,
                 precision: int = B.DPP_FP64, device: str | torch.device = "cuda",
                 cell_kind: int = 0):
        if not torch.cuda.is_available():
            raise RuntimeError("DPPSystem needs a CUDA device; libdpp has no CPU fallback")
        self.device = torch.device(device)
        self.dim = int(np.asarray(coords).shape[1]) if not isinstance(coords, torch.Tensor) \
            else int(coords.shape[1])
        self.coords = _dev(coords, torch.float64, self.device)
        self.cells = _dev(cells, torch.int32, self.device)
        self.bfacets = _dev(bfacets, torch.int32, self.device)
        self.log_k1 = _dev(log_k1, torch.float64, self.device)
        self.log_k2 = _dev(log_k2, torch.float64, self.device)
        self.p01 = _dev(p01, torch.float64, self.device)
        self.p02 = _dev(p02, torch.float64, self.device)
        self.mu = float(mu)
        self.beta = float(beta)
        gb = list(np.asarray(gamma_b, dtype=np.float64).ravel()) + [0.0] * 3
        self.gamma_b = gb[:3]
        self.precision = precision
        self.cell_kind = int(cell_kind)
        self.n_nodes = int(self.coords.shape[0])
        self.n_cells = int(self.cells.shape[0])
        self.ns = 2 * self.dim + 2
        self.prob = 0
        self.pc = 0
        self.desc = self._desc()
        self.prob = B.dpp_assemble(self.desc, precision, _stream(self.device))

    @classmethod
    def from_problem(cls, p, precision: int = B.DPP_FP64, device="cuda"):
        m = p.mesh
        kind = B.DPP_CELL_Q1 if getattr(m, "kind", "simplex") == "q1" else B.DPP_CELL_SIMPLEX
        return cls(m.coords, m.cells, m.bfacets, p.logk1, p.logk2, p.mu, p.beta, p.gamma_b, p.p01,
                   p.p02, precision=precision, device=device, cell_kind=kind)

    def _desc(self) -> B.dpp_problem_desc:
        d = B.dpp_problem_desc()
        d.dim = self.dim
        d.memory = B.DPP_MEM_DEVICE
        d.n_nodes = self.n_nodes
        d.n_cells = self.n_cells
        d.n_bfacets = int(self.bfacets.shape[0])
        d.coords = self.coords.data_ptr()
        d.cells = self.cells.data_ptr()
        d.bfacets = self.bfacets.data_ptr() if d.n_bfacets else None
        d.log_k1 = self.log_k1.data_ptr()
        d.log_k2 = self.log_k2.data_ptr()
        d.mu = self.mu
        d.beta = self.beta
        for k in range(3):
            d.gamma_b[k] = self.gamma_b[k]
        d.p01 = self.p01.data_ptr()
        d.p02 = self.p02.data_ptr()
        d.cell_kind = self.cell_kind
        return d

    # ------------------------------------------------------------------ pc / solve
    def setup_pc(self, **opts) -> "DPPSystem":
        o = B.dpp_pc_opts_default()
        for k, v in opts.items():
            setattr(o, k, v)
        if self.pc:
            B.dpp_destroy_pc(self.pc)
            self.pc = 0
        self.pc = B.dpp_setup_pc(self.prob, o, _stream(self.device))
        return self

    def solve_opts(self, **opts) -> B.dpp_solve_opts:
        o = B.dpp_solve_opts_default()
        for k, v in opts.items():
            setattr(o, k, v)
        return o

    def solve(self, x0: torch.Tensor | None = None, check: bool = True, **opts):
        """Solve K x = f. Returns (x [n_nodes, 2d+2] float64 on the device, info dict)."""
        if not self.pc:
            self.setup_pc()
        o = self.solve_opts(**opts)
        if x0 is not None:
            x = x0.to(self.device, torch.float64).contiguous().clone()
            o.x0_zero = 0
        else:
            x = torch.zeros((self.n_nodes, self.ns), dtype=torch.float64, device=self.device)
        allow = (B.DPP_OK,) if check else tuple(range(9))
        info = B.dpp_solve(self.prob, self.pc, o, x, _stream(self.device), allow=allow)
        return x, info.as_dict()

    def solve_rhs(self, b: torch.Tensor, check: bool = True, **opts):
        """Solve K x = b for a given right-hand side (x0 = 0). Returns (x, info)."""
        if not self.pc:
            self.setup_pc()
        o = self.solve_opts(**opts)
        b = b.to(self.device, torch.float64).contiguous()
        x = torch.zeros_like(b)
        allow = (B.DPP_OK,) if check else tuple(range(9))
        info = B.dpp_solve_rhs(self.prob, self.pc, o, b, x, _stream(self.device), allow=allow)
        return x, info.as_dict()

    def adjoint(self, x: torch.Tensor, dJdx: torch.Tensor, check: bool = True, **opts):
        """Adjoint solve: (lambda, dJ/dlogk1, dJ/dlogk2, dJ/dbeta, info)."""
        if not self.pc:
            self.setup_pc()
        o = self.solve_opts(**opts)
        x = x.to(self.device, torch.float64).contiguous()
        g = dJdx.to(self.device, torch.float64).contiguous()
        lam = torch.zeros_like(g)
        g1 = torch.empty(self.n_cells, dtype=torch.float64, device=self.device)
        g2 = torch.empty_like(g1)
        gb = torch.empty(1, dtype=torch.float64, device=self.device)
        allow = (B.DPP_OK,) if check else tuple(range(9))
        info = B.dpp_adjoint_solve(self.prob, self.pc, o, x, g, lam, g1, g2, gb,
                                   _stream(self.device), allow=allow)
        return lam, g1, g2, gb, info.as_dict()

    # ------------------------------------------------------------------ inspection
    def sizes(self) -> dict:
        return B.dpp_problem_sizes(self.prob)

    def apply_K(self, x: torch.Tensor, transpose: bool = False) -> torch.Tensor:
        x = x.to(self.device, torch.float64).contiguous()
        y = torch.empty_like(x)
        B.dpp_apply_K(self.prob, transpose, x, y, _stream(self.device))
        return y

    def apply_K32(self, x: torch.Tensor, transpose: bool = False) -> torch.Tensor:
        x = x.to(self.device, torch.float32).contiguous()
        y = torch.empty(x.shape, dtype=torch.float64, device=self.device)
        B.dpp_apply_K32(self.prob, transpose, x, y, _stream(self.device))
        return y

    def apply_K_mf(self, x: torch.Tensor, transpose: bool = False) -> torch.Tensor:
        x = x.to(self.device, torch.float64).contiguous()
        y = torch.empty_like(x)
        B.dpp_apply_K_mf(self.prob, transpose, x, y, _stream(self.device))
        return y

    def apply_K32_mf(self, x: torch.Tensor, transpose: bool = False) -> torch.Tensor:
        x = x.to(self.device, torch.float32).contiguous()
        y = torch.empty(x.shape, dtype=torch.float64, device=self.device)
        B.dpp_apply_K32_mf(self.prob, transpose, x, y, _stream(self.device))
        return y

    def rhs(self) -> torch.Tensor:
        f = torch.empty((self.n_nodes, self.ns), dtype=torch.float64, device=self.device)
        B.dpp_get_rhs(self.prob, f, _stream(self.device))
        return f

    def export_pairs(self):
        s = self.sizes()
        rp = torch.empty(self.n_nodes + 1, dtype=torch.int32, device=self.device)
        col = torch.empty(s["n_pairs"], dtype=torch.int32, device=self.device)
        vals = torch.empty((s["n_pairs"], s["values_per_pair"]), dtype=torch.float64,
                           device=self.device)
        B.dpp_export_pairs(self.prob, rp, col, vals, _stream(self.device))
        return rp, col, vals

    def pc_apply(self, r: torch.Tensor, transpose: bool = False) -> torch.Tensor:
        if not self.pc:
            self.setup_pc()
        r = r.to(self.device, torch.float64).contiguous()
        z = torch.empty_like(r)
        B.dpp_pc_apply(self.prob, self.pc, transpose, r, z, _stream(self.device))
        return z

    def pc_apply_mass(self, r: torch.Tensor) -> torch.Tensor:
        r = r.to(self.device, torch.float64).contiguous()
        z = torch.empty_like(r)
        B.dpp_pc_apply_mass(self.prob, self.pc, r, z, _stream(self.device))
        return z

    def hierarchies(self) -> int:
        return B.dpp_pc_hierarchies(self.pc)

    def level(self, level: int, with_p: bool = True, hierarchy: int = 0):
        s = B.dpp_pc_level_sizes(self.pc, level, hierarchy)
        dev = self.device
        rp = torch.empty(s["rows"] + 1, dtype=torch.int32, device=dev)
        col = torch.empty(max(s["nnz"], 1), dtype=torch.int32, device=dev)
        val = torch.empty(max(s["nnz"], 1), dtype=torch.float64, device=dev)
        prp = pcol = pval = None
        if with_p and s["p_cols"]:
            prp = torch.empty(s["rows"] + 1, dtype=torch.int32, device=dev)
            pcol = torch.empty(s["p_nnz"], dtype=torch.int32, device=dev)
            pval = torch.empty(s["p_nnz"], dtype=torch.float64, device=dev)
        B.dpp_pc_export_level(self.pc, level, rp, col, val, prp, pcol, pval, _stream(dev),
                              hierarchy=hierarchy)
        return s, (rp, col[:s["nnz"]], val[:s["nnz"]]), (prp, pcol, pval)

    def close(self):
        if self.pc:
            B.dpp_destroy_pc(self.pc)
            self.pc = 0
        if self.prob:
            B.dpp_destroy_problem(self.prob)
            self.prob = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class DPPSolve(torch.autograd.Function):
    """x = K(log k1, log k2, beta)^-1 f, differentiable through the hand-written adjoint.

    forward(log_k1 [n_cells], log_k2 [n_cells], beta [1], mesh, opts) -> x [n_nodes, 2d+2].
    ``mesh`` is a dict with coords, cells, bfacets, mu, gamma_b, p01, p02. The
    backward pass calls dpp_adjoint_solve with the same preconditioner.
    """

    @staticmethod
    def forward(ctx, log_k1, log_k2, beta, mesh, opts=None):
        opts = opts or {}
        sysm = DPPSystem(mesh["coords"], mesh["cells"], mesh["bfacets"], log_k1.detach(),
                         log_k2.detach(), mesh["mu"], float(beta.detach().reshape(-1)[0]),
                         mesh["gamma_b"], mesh["p01"], mesh["p02"], device=log_k1.device)
        sysm.setup_pc(**opts.get("pc", {}))
        x, info = sysm.solve(**opts.get("solve", {}))
        ctx.system = sysm
        ctx.opts = opts
        ctx.save_for_backward(x)
        ctx.info = info
        return x

    @staticmethod
    def backward(ctx, grad_x):
        (x,) = ctx.saved_tensors
        sysm = ctx.system
        _, g1, g2, gb, _ = sysm.adjoint(x, grad_x.contiguous(), **ctx.opts.get("solve", {}))
        sysm.close()
        return g1, g2, gb.reshape(1), None, None


class DPPBatch:
    """Device-resident inputs of many problems for dpp_solve_batched.

    ``problems``: objects with the fields of a problem description (mesh with
    coords/cells/bfacets, logk1, logk2, mu, beta, gamma_b, p01, p02).
    """

    def __init__(self, problems, device="cuda"):
        self.device = torch.device(device)
        dev = self.device
        self.keep, self.descs, self.xs = [], [], []
        for p in problems:
            m = p.mesh
            t = dict(coords=_dev(m.coords, torch.float64, dev), cells=_dev(m.cells, torch.int32, dev),
                     bfacets=_dev(m.bfacets, torch.int32, dev),
                     log_k1=_dev(p.logk1, torch.float64, dev),
                     log_k2=_dev(p.logk2, torch.float64, dev), p01=_dev(p.p01, torch.float64, dev),
                     p02=_dev(p.p02, torch.float64, dev))
            self.keep.append(t)
            d = B.dpp_problem_desc()
            d.dim = int(m.coords.shape[1])
            d.memory = B.DPP_MEM_DEVICE
            d.n_nodes = int(m.coords.shape[0])
            d.n_cells = int(m.cells.shape[0])
            d.n_bfacets = int(m.bfacets.shape[0])
            for k in ("coords", "cells", "bfacets", "log_k1", "log_k2", "p01", "p02"):
                setattr(d, k, t[k].data_ptr() if t[k].numel() else None)
            d.mu, d.beta = float(p.mu), float(p.beta)
            d.cell_kind = B.DPP_CELL_Q1 if getattr(m, "kind", "simplex") == "q1" else 0
            gb = list(np.asarray(p.gamma_b, dtype=np.float64).ravel()) + [0.0] * 3
            for k in range(3):
                d.gamma_b[k] = gb[k]
            self.descs.append(d)
            self.xs.append(torch.zeros((d.n_nodes, 2 * d.dim + 2), dtype=torch.float64, device=dev))
        self.n_dofs = sum(int(x.numel()) for x in self.xs)

    def solve(self, precision: int = B.DPP_FP64, pc_opts: dict | None = None, **solve_opts):
        """Returns (list of x tensors, list of per-instance info dicts, status)."""
        po = B.dpp_pc_opts_default()
        po.precision = precision
        for k, v in (pc_opts or {}).items():
            setattr(po, k, v)
        so = B.dpp_solve_opts_default()
        for k, v in solve_opts.items():
            setattr(so, k, v)
        st, infos = B.dpp_solve_batched(self.descs, po, so, self.xs, _stream(self.device),
                                        allow=tuple(range(9)))
        return self.xs, infos, st


def solve_batched(problems, precision: int = B.DPP_FP64, device="cuda", pc_opts: dict | None = None,
                  **solve_opts):
    """One-shot batched solve; see DPPBatch."""
    return DPPBatch(problems, device).solve(precision, pc_opts, **solve_opts)

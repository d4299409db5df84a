"""PyTorch-facing wrapper: tensors in, tensors out; all work in libsfairsc.so.

PyTorch provides device memory and the stream; every computation is a call
into the C ABI (see include/sfairsc.h).
"""
from __future__ import annotations

import torch

from . import binding as B

_DTYPES = {torch.float64: B.SFAIRSC_F64, torch.float32: B.SFAIRSC_F32, torch.bfloat16: B.SFAIRSC_BF16}


def _ptr(t: torch.Tensor | None):
    return None if t is None else t.data_ptr()


class FairSC:
    """One graph's s-FairSC context (Algorithm 3).

    row_ptr, col_idx: int32 CSR of the symmetric weight matrix W (both triangles);
    values: float64 / float32 / bfloat16 weights; groups: int32 labels in [0, h).
    Tensors may live on the GPU (borrowed: keep them alive) or the CPU (copied).
    F: a dense float64 constraint matrix (n x p) in place of the groups (pass groups=None);
    the constraint is then F^T H = 0 (sfairsc_create_dense).
    """

    def __init__(self, row_ptr, col_idx, values, groups, k: int, h: int | None = None, normalized: bool = True,
                 prec: str = "mixed", block: int = 1, tol: float = 1e-6, basis: int = 0, max_restarts: int = 200,
                 sigma: float | None = None, seed: int = 1, kmeans_seed: int = 0, kmeans_n_init: int = 1,
                 kmeans_max_iter: int = 100, validate: int = 1, profile: int = 0, wait_limit_us: int = 0,
                 fault_inject: int = 0, spmv_window: int = 0, orth_mode: int = 0, restart_mode: int = 0,
                 stream: torch.cuda.Stream | None = None, F: torch.Tensor | None = None):
        if F is not None:
            F = F.to(torch.float64).contiguous()
            groups = torch.zeros(row_ptr.numel() - 1, dtype=torch.int32, device=row_ptr.device)
        self._keep = [t.contiguous() for t in (row_ptr, col_idx, values, groups)]
        row_ptr, col_idx, values, groups = self._keep
        if F is not None:
            self._keep.append(F)
        if row_ptr.dtype != torch.int32 or col_idx.dtype != torch.int32 or groups.dtype != torch.int32:
            raise TypeError("row_ptr, col_idx and groups must be int32")
        if values.dtype not in _DTYPES:
            raise TypeError("values must be float64, float32 or bfloat16")
        self.n = row_ptr.numel() - 1
        self.nnz = col_idx.numel()
        self.k = int(k)
        if F is not None:
            self.h = F.shape[1] + 1
        else:
            self.h = int(h) if h is not None else int(groups.max().item()) + 1
        self.prec = prec
        self.vec_dtype = torch.float64 if prec == "fp64" else torch.float32
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        opts = B.make_opts(prec, block, tol, basis, max_restarts, sigma, seed, kmeans_seed, kmeans_n_init,
                           kmeans_max_iter, validate, profile, wait_limit_us, fault_inject, spmv_window, orth_mode,
                           restart_mode)
        if F is not None:
            self.ctx = B.sfairsc_create_dense(self.n, self.nnz, _ptr(row_ptr), _ptr(col_idx), _ptr(values),
                                              _DTYPES[values.dtype], _ptr(F), F.shape[1], self.k,
                                              1 if normalized else 0, opts, self.stream.cuda_stream)
        else:
            self.ctx = B.sfairsc_create(self.n, self.nnz, _ptr(row_ptr), _ptr(col_idx), _ptr(values),
                                        _DTYPES[values.dtype], _ptr(groups), self.h, self.k, 1 if normalized else 0,
                                        opts, self.stream.cuda_stream)
        self.sigma = B.sfairsc_get_sigma(self.ctx)
        self.info = None

    def close(self):
        if getattr(self, "ctx", None):
            B.sfairsc_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def apply_operator(self, w: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        """L_n^sigma w for w of shape (n,) or (n, b), b <= 4 (Sec. 3.4 (i))."""
        vec = w.dim() == 1
        W = w.reshape(self.n, -1)
        nv = W.shape[1]
        Wc = W.t().contiguous().to(self.vec_dtype)  # column-major: each vector contiguous
        O = torch.empty_like(Wc) if out is None else out.view(nv, self.n)
        B.sfairsc_apply_operator(self.ctx, _ptr(Wc), _ptr(O), nv)
        res = O.t()
        return res.reshape(-1) if vec else res

    def solve(self, want_labels: bool = True, allow_not_converged: bool = False, on_host: bool = False,
              out: tuple | None = None):
        """Eigenvalues (k,), H (n, k) and labels (n,) plus the info dict.  out = (lam, H, labels)
        writes into caller-owned tensors (float64 (k,), float64 (n, k), int32 (n,) or None; host or
        device, contiguous), e.g. pinned host buffers allocated once for repeated solves."""
        if out is not None:
            lam, H, lab = out
            if lam.dtype != torch.float64 or lam.numel() != self.k or not lam.is_contiguous():
                raise ValueError("out[0] must be a contiguous float64 tensor of k values")
            if H.dtype != torch.float64 or H.shape != (self.n, self.k) or not H.is_contiguous():
                raise ValueError("out[1] must be a contiguous float64 (n, k) tensor")
            if lab is not None and (lab.dtype != torch.int32 or lab.numel() != self.n or not lab.is_contiguous()):
                raise ValueError("out[2] must be a contiguous int32 tensor of n values")
        else:
            dev = torch.device("cpu") if on_host else self.device
            lam = torch.empty(self.k, dtype=torch.float64, device=dev)
            H = torch.empty(self.n, self.k, dtype=torch.float64, device=dev)
            lab = torch.empty(self.n, dtype=torch.int32, device=dev) if want_labels else None
            if on_host:
                lam, H = lam.pin_memory(), H.pin_memory()
                lab = lab.pin_memory() if lab is not None else None
        allow = (0, -7) if allow_not_converged else (0,)
        rc, info = B.sfairsc_solve(self.ctx, _ptr(lam), _ptr(H), _ptr(lab), allow)
        self.info = info.as_dict()
        self.status = rc
        return lam, H, lab, self.info

    def backward_vectors(self, grad_H: torch.Tensor, grad_lambda: torch.Tensor | None = None,
                         bandwidth: float | None = None, max_iter: int = 0, rtol: float = 0.0):
        """d loss / d values (nnz,) for a loss on H (grad_H = d loss / d H, n x k) and optionally on the
        eigenvalues; also d / d bandwidth, the CG iterations and the final relative residual."""
        G = grad_H.to(device=self.device, dtype=torch.float64).contiguous()
        gl = None if grad_lambda is None else grad_lambda.to(device=self.device, dtype=torch.float64).contiguous()
        out = torch.empty(self.nnz, dtype=torch.float64, device=self.device)
        gs, it, rr = B.sfairsc_backward_vectors(self.ctx, _ptr(G), _ptr(gl), _ptr(out), bandwidth or 0.0,
                                                want_bandwidth=bandwidth is not None, max_iter=max_iter, rtol=rtol)
        return out, gs, it, rr

    def backward(self, grad_lambda: torch.Tensor, bandwidth: float | None = None):
        """d(sum_i gbar_i lambda_i)/d values (nnz,) and optionally d/d bandwidth."""
        g = grad_lambda.to(device=self.device, dtype=torch.float64).contiguous()
        out = torch.empty(self.nnz, dtype=torch.float64, device=self.device)
        gs = B.sfairsc_backward(self.ctx, _ptr(g), _ptr(out), bandwidth or 0.0, want_bandwidth=bandwidth is not None)
        return out, gs


def kmeans(H: torch.Tensor, k: int, seed: int = 0, n_init: int = 1, max_iter: int = 100):
    """Seeded, exactly reproducible k-means on the rows of H (labels, centroids, inertia, iterations)."""
    X = H.to(torch.float64).contiguous()
    n, d = X.shape
    lab = torch.empty(n, dtype=torch.int32, device=X.device)
    cen = torch.empty(k, d, dtype=torch.float64, device=X.device)
    stream = torch.cuda.current_stream().cuda_stream if X.is_cuda else None
    inertia, iters = B.sfairsc_kmeans(n, d, _ptr(X), k, seed, n_init, max_iter, _ptr(lab), _ptr(cen), stream)
    return lab, cen, inertia, iters


class FairEigenvalueSum(torch.autograd.Function):
    """lambda_1..lambda_k of the fair problem as a differentiable function of the edge weights.

    forward(values, row_ptr, col_idx, groups, k, h, bandwidth, opts) -> eigenvalues (k,)
    backward gives d/d values through the SDDMM kernel and, when bandwidth is
    a tensor, d/d bandwidth for Gaussian weights w = exp(-r^2 / (2 s^2)).
    """

    @staticmethod
    def forward(ctx, values, row_ptr, col_idx, groups, k, h, bandwidth=None, opts=None):
        opts = dict(opts or {})
        solver = FairSC(row_ptr, col_idx, values.detach(), groups, k, h, **opts)
        lam, H, _, info = solver.solve(want_labels=False, allow_not_converged=True)
        ctx.solver = solver
        ctx.has_bw = isinstance(bandwidth, torch.Tensor)
        ctx.bw = float(bandwidth) if ctx.has_bw else None
        ctx.values_dtype = values.dtype
        return lam

    @staticmethod
    def backward(ctx, grad_lam):
        gv, gs = ctx.solver.backward(grad_lam, ctx.bw)
        ctx.solver.close()
        gbw = torch.tensor(gs, dtype=torch.float64, device=gv.device) if ctx.has_bw else None
        return gv.to(ctx.values_dtype), None, None, None, None, None, gbw, None


class FairEmbedding(torch.autograd.Function):
    """(eigenvalues, H) of the fair problem as a differentiable function of the edge weights.

    forward(values, row_ptr, col_idx, groups, k, h, bandwidth, opts) -> (eigenvalues (k,), H (n, k))
    backward: d/d values (and d/d bandwidth) of any loss on both outputs, through the
    eigenvector-level backward (conjugate-gradient solves and an SDDMM in the library).
    """

    @staticmethod
    def forward(ctx, values, row_ptr, col_idx, groups, k, h, bandwidth=None, opts=None):
        opts = dict(opts or {})
        solver = FairSC(row_ptr, col_idx, values.detach(), groups, k, h, **opts)
        lam, H, _, info = solver.solve(want_labels=False, allow_not_converged=True)
        ctx.solver = solver
        ctx.has_bw = isinstance(bandwidth, torch.Tensor)
        ctx.bw = float(bandwidth) if ctx.has_bw else None
        ctx.values_dtype = values.dtype
        return lam, H

    @staticmethod
    def backward(ctx, grad_lam, grad_H):
        if grad_H is None:
            grad_H = torch.zeros(ctx.solver.n, ctx.solver.k, dtype=torch.float64, device=ctx.solver.device)
        gv, gs, _, _ = ctx.solver.backward_vectors(grad_H, grad_lam, ctx.bw)
        ctx.solver.close()
        gbw = torch.tensor(gs, dtype=torch.float64, device=gv.device) if ctx.has_bw else None
        return gv.to(ctx.values_dtype), None, None, None, None, None, gbw, None


class FairSCBatch:
    """Many s-FairSC eigenproblems solved by one persistent launch (batched form).

    graphs: sequence of dicts with row_ptr, col_idx (int32), values (float32),
    groups (int32) CUDA tensors and k, h.  Inputs are borrowed (kept alive
    here); eigenvalues and H are allocated per graph on the device.
    """

    def __init__(self, graphs, tol: float = 1e-6, basis: int = 0, max_restarts: int = 200, seed: int = 1,
                 validate: int = 1, want_H: bool = True, autotune: bool = False,
                 stream: torch.cuda.Stream | None = None):
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._keep = []
        self.lam, self.H, descs = [], [], []
        for g in graphs:
            rp, ci, va, gr = (g[key].contiguous() for key in ("row_ptr", "col_idx", "values", "groups"))
            if rp.dtype != torch.int32 or ci.dtype != torch.int32 or gr.dtype != torch.int32:
                raise TypeError("row_ptr, col_idx and groups must be int32")
            if va.dtype != torch.float32:
                raise TypeError("batched values must be float32")
            if not all(t.is_cuda for t in (rp, ci, va, gr)):
                raise ValueError("batched inputs must be CUDA tensors")
            self._keep += [rp, ci, va, gr]
            n, k, h = rp.numel() - 1, int(g["k"]), int(g["h"])
            lam = torch.empty(k, dtype=torch.float64, device=self.device)
            H = torch.empty(n, k, dtype=torch.float64, device=self.device) if want_H else None
            self.lam.append(lam)
            self.H.append(H)
            descs.append(B.BatchGraph(n, ci.numel(), _ptr(rp), _ptr(ci), _ptr(va), _ptr(gr), h, k, _ptr(lam),
                                      _ptr(H) if H is not None else None))
        self.count = len(descs)
        opts = B.make_opts("mixed", 4, tol, basis, max_restarts, None, seed, validate=validate)
        self.handle = B.sfairsc_batch_create(descs, opts, self.stream.cuda_stream)
        if autotune:
            B.sfairsc_batch_autotune(self.handle)

    def solve(self, allow_not_converged: bool = False):
        """Returns (status list, info dict); results are in self.lam / self.H."""
        allow = (0, -7) if allow_not_converged else (0,)
        _, status, info = B.sfairsc_batch_solve(self.handle, self.count, allow=allow)
        return status, info.as_dict()

    def stats(self):
        """Per-graph restarts, matvecs and residuals of the last solve."""
        return B.sfairsc_batch_stats(self.handle, self.count)

    def close(self):
        if getattr(self, "handle", None):
            B.sfairsc_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

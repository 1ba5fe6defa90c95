"""ctypes binding of the kx C ABI (include/kx.h).

Argument marshalling only: every numerical step runs in libkx.so's CUDA
kernels.  PyTorch supplies device memory and the CUDA stream.  There is no
CPU fallback: without the built library every call raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(HERE, "libkx.so")

KX_OK, KX_EINVAL, KX_ENOMEM, KX_ECUDA, KX_ENONFINITE, KX_ENOCONV, KX_ETIMEOUT = range(7)
KX_PERIODIC, KX_PEC = 0, 1
KX_FP64, KX_FP32 = 0, 1
KX_PLAIN, KX_SPLIT, KX_RSTDIM, KX_SPLIT2, KX_SPLIT4D = 0, 1, 2, 3, 4
METHODS = {"plain": KX_PLAIN, "split": KX_SPLIT, "rstdim": KX_RSTDIM, "split2": KX_SPLIT2,
           "split4d": KX_SPLIT4D}
STATUS_NAMES = {0: "KX_OK", 1: "KX_EINVAL", 2: "KX_ENOMEM", 3: "KX_ECUDA",
                4: "KX_ENONFINITE", 5: "KX_ENOCONV", 6: "KX_ETIMEOUT"}

EXPORTS = ["krylov_expm_create", "krylov_expm_create_mat", "krylov_expm_destroy", "kx_num_unknowns", "apply_A",
           "arnoldi", "expm_phi_project", "stationary_solve", "expm_action",
           "response_at_freqs", "kx_get_stats", "kx_reset_stats", "kx_set_timing",
           "kx_kernel_times", "kx_last_error", "kx_arnoldi_noalloc", "kx_noalloc_last_error",
           "adjoint_response_grad", "kx_set_permittivity", "response_at_freqs_multi", "kx_stream",
           "response_restart_dim", "kx_wait_selftest", "kx_batch_create", "kx_batch_destroy",
           "kx_batch_get_info", "kx_batch_last_error", "response_restart_dim_batch", "kx_batch_set_timing"]
KCLASSES = ["pass_a", "pass_b", "restart", "projected", "zupdate", "apply", "cascade", "sweep", "swapply"]
# Arnoldi forms (kx_desc.arnoldi_form)
ARNOLDI_FORMS = {"default": 0, "twopass": 1, "sweep": 2}


class KxError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Desc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("bc", ctypes.c_int * 3),
                ("layer_axis", ctypes.c_int), ("layer_cells", ctypes.c_int),
                ("sigma_max", ctypes.c_double), ("precision", ctypes.c_int),
                ("krylov_dim", ctypes.c_int), ("max_freqs", ctypes.c_int), ("batch", ctypes.c_int),
                ("max_checkpoints", ctypes.c_int), ("rst_samples", ctypes.c_int), ("pml", ctypes.c_int),
                ("arnoldi_form", ctypes.c_int)]


class KernelTime(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double), ("bytes", ctypes.c_double), ("launches", ctypes.c_int64)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("problems", ctypes.c_int), ("sweep_tiles_per_block", ctypes.c_int),
                ("apply_rounds_per_thread", ctypes.c_int), ("sweep_blocks", ctypes.c_int),
                ("apply_blocks", ctypes.c_int), ("from_cache", ctypes.c_int), ("tune_ms", ctypes.c_double),
                ("batched_launches", ctypes.c_int64), ("sweep_ms", ctypes.c_double), ("sweep_bytes", ctypes.c_double),
                ("sweep_timed_launches", ctypes.c_int64), ("graph_replays", ctypes.c_int64)]


class Stats(ctypes.Structure):
    _fields_ = [("matvecs", ctypes.c_int64), ("arnoldi_steps", ctypes.c_int64),
                ("substeps", ctypes.c_int64), ("expm_evals", ctypes.c_int64),
                ("fom_cycles", ctypes.c_int64), ("kernel_launches", ctypes.c_int64)]


_lib = None


def load_library(path: Optional[str] = None):
    """Load libkx.so; raise if it is not built (no fallback exists)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIBPATH
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is not built: run `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(p)
    vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
    lib.krylov_expm_create.argtypes = [ctypes.POINTER(Desc), dp, vp, ctypes.POINTER(vp)]
    lib.krylov_expm_create_mat.argtypes = [ctypes.POINTER(Desc), vp, dp, ctypes.c_int, vp, ctypes.POINTER(vp)]
    lib.krylov_expm_destroy.argtypes = [vp]
    lib.kx_num_unknowns.argtypes = [vp]
    lib.kx_num_unknowns.restype = ctypes.c_int64
    lib.kx_stream.argtypes = [vp]
    lib.kx_stream.restype = vp
    lib.apply_A.argtypes = [vp, vp, vp, ctypes.c_int]
    lib.arnoldi.argtypes = [vp, vp, ctypes.c_int, vp, vp, dp, ip]
    lib.expm_phi_project.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                     ctypes.c_double, dp, ctypes.c_int, vp]
    lib.stationary_solve.argtypes = [vp, vp, dp, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                     vp, vp, dp, ip]
    lib.expm_action.argtypes = [vp, vp, ctypes.c_double, ctypes.c_double, vp, dp]
    lib.response_at_freqs.argtypes = [vp, vp, dp, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_int, ip, vp, dp, dp, vp]
    lib.response_restart_dim.argtypes = [vp, vp, dp, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_int, ip, vp, dp, dp, ip, vp]
    lib.kx_get_stats.argtypes = [vp, ctypes.POINTER(Stats)]
    lib.kx_reset_stats.argtypes = [vp]
    lib.adjoint_response_grad.argtypes = [vp, vp, dp, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                          ip, vp, dp]
    lib.kx_set_permittivity.argtypes = [vp, vp]
    lib.response_at_freqs_multi.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(vp), dp,
                                            ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, ip,
                                            dp, dp, ctypes.c_int]
    lib.kx_set_timing.argtypes = [vp, ctypes.c_int]
    lib.kx_kernel_times.argtypes = [vp, ctypes.POINTER(KernelTime)]
    lib.kx_last_error.argtypes = [vp]
    lib.kx_last_error.restype = ctypes.c_char_p
    lib.kx_arnoldi_noalloc.argtypes = [ctypes.POINTER(Desc), vp, vp, ctypes.c_int, vp, vp, dp, ip, vp]
    lib.kx_noalloc_last_error.argtypes = []
    lib.kx_wait_selftest.argtypes = [vp, ctypes.c_uint]
    lib.kx_noalloc_last_error.restype = ctypes.c_char_p
    lib.kx_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, vp, ctypes.POINTER(vp)]
    lib.kx_batch_destroy.argtypes = [vp]
    lib.kx_batch_get_info.argtypes = [vp, ctypes.POINTER(BatchInfo)]
    lib.kx_batch_set_timing.argtypes = [vp, ctypes.c_int]
    lib.kx_batch_last_error.argtypes = [vp]
    lib.kx_batch_last_error.restype = ctypes.c_char_p
    lib.response_restart_dim_batch.argtypes = [vp, ctypes.POINTER(vp), dp, ctypes.c_int, ctypes.c_double,
                                               ctypes.c_double, ctypes.c_int, ip, dp, dp, ip]
    for name in EXPORTS:
        if name not in ("kx_num_unknowns", "kx_last_error", "kx_noalloc_last_error", "kx_stream",
                        "kx_batch_last_error"):
            getattr(lib, name).restype = ctypes.c_int
    if path is None:
        _lib = lib
    return lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Context:
    """One solver context: grid, permittivity, precision and workspace.

    ``grid`` is any object with attributes dim, n, bc, layer_axis,
    layer_cells, sigma_max and optionally pml (e.g. ``scenario.Grid``).  ``eps_cell`` is the
    per-cell permittivity (numpy, x fastest).  ``stream``: a torch CUDA
    stream (default: the current stream), or ``"own"`` for a private stream
    created by the library (distinct per context; use it for concurrent
    problems, since torch hands out streams from a small pool).
    ``rst_samples``: time samples per frequency held for the restart-in-
    dimension method (``method="rstdim"``; 0 leaves it unavailable).
    ``arnoldi``: "default" (single sweep for restart in dimension on grids of
    3e6 unknowns or more, two passes elsewhere), "twopass" or "sweep" (also
    for ``arnoldi()``).
    ``mat_id`` / ``eps_table``: instead of ``eps_cell`` (pass None), a CUDA
    uint8 tensor of material ids per cell and the materials' permittivities
    (``krylov_expm_create_mat``).
    """

    def __init__(self, grid, eps_cell, precision: str = "fp32", krylov_dim: int = 64,
                 max_freqs: int = 1, batch: int = 1, stream=None, max_checkpoints: int = 0,
                 rst_samples: int = 0, arnoldi: str = "default", mat_id=None, eps_table=None):
        import torch
        self._torch = torch
        self.lib = load_library()
        self.grid = grid
        d = Desc()
        d.dim = grid.dim
        n = list(grid.n) + [1] * (3 - len(grid.n))
        bc = list(grid.bc) + [0] * (3 - len(grid.bc))
        d.n = (ctypes.c_int * 3)(*n)
        d.bc = (ctypes.c_int * 3)(*bc)
        d.layer_axis = grid.layer_axis
        d.layer_cells = grid.layer_cells
        d.sigma_max = grid.sigma_max
        d.precision = KX_FP64 if precision == "fp64" else KX_FP32
        d.krylov_dim = krylov_dim
        d.max_freqs = max_freqs
        d.batch = batch
        d.max_checkpoints = max_checkpoints
        d.rst_samples = rst_samples
        d.pml = int(getattr(grid, "pml", 0))
        if arnoldi not in ARNOLDI_FORMS:
            raise ValueError(f"arnoldi must be one of {sorted(ARNOLDI_FORMS)}")
        d.arnoldi_form = ARNOLDI_FORMS[arnoldi]
        self.desc = d
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        own = isinstance(stream, str) and stream == "own"
        self.stream = None if own else (stream if stream is not None else torch.cuda.current_stream())
        h = ctypes.c_void_p()
        sarg = ctypes.c_void_p(-1) if own else ctypes.c_void_p(self.stream.cuda_stream)
        if eps_cell is None:
            if not (isinstance(mat_id, torch.Tensor) and mat_id.is_cuda and mat_id.dtype == torch.uint8):
                raise TypeError("mat_id must be a CUDA uint8 tensor")
            mid = mat_id.contiguous()
            tab = np.ascontiguousarray(np.asarray(eps_table, np.float64).reshape(-1))
            st = self.lib.krylov_expm_create_mat(ctypes.byref(d), ctypes.c_void_p(mid.data_ptr()), _dptr(tab),
                                                 len(tab), sarg, ctypes.byref(h))
        else:
            eps = np.ascontiguousarray(np.asarray(eps_cell, np.float64).reshape(-1))
            st = self.lib.krylov_expm_create(ctypes.byref(d), _dptr(eps), sarg, ctypes.byref(h))
        if st != KX_OK:
            raise KxError(st, self.lib.kx_last_error(None).decode())
        self.h = h
        self.n = int(self.lib.kx_num_unknowns(h))
        if own:
            self.stream = torch.cuda.ExternalStream(int(self.lib.kx_stream(h)))

    # -- helpers -----------------------------------------------------------
    def _check(self, st):
        if st != KX_OK:
            raise KxError(st, self.lib.kx_last_error(self.h).decode())

    def _vec(self, t, name, ncols=1):
        torch = self._torch
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise TypeError(f"{name} must be a CUDA tensor")
        if t.dtype != self.dtype:
            raise TypeError(f"{name} must be {self.dtype}")
        if not t.is_contiguous() or t.numel() != self.n * ncols:
            raise ValueError(f"{name} must be contiguous with {self.n * ncols} elements")
        return ctypes.c_void_p(t.data_ptr())

    def empty(self, *cols):
        return self._torch.empty((*cols, self.n), dtype=self.dtype, device="cuda")

    def close(self):
        if getattr(self, "h", None):
            self.lib.krylov_expm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def stats(self):
        s = Stats()
        self._check(self.lib.kx_get_stats(self.h, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in Stats._fields_}

    def reset_stats(self):
        self._check(self.lib.kx_reset_stats(self.h))

    def set_timing(self, on: bool):
        self._check(self.lib.kx_set_timing(self.h, int(bool(on))))

    def wait_selftest(self, rounds: int = 1000) -> int:
        """Run the library's bounded device wait on an mbarrier nothing
        completes; returns the status (KX_ETIMEOUT expected), no raise."""
        return int(self.lib.kx_wait_selftest(self.h, rounds))

    def kernel_times(self):
        """Per-class {ms, bytes, launches} recorded since timing was switched on."""
        arr = (KernelTime * len(KCLASSES))()
        self._check(self.lib.kx_kernel_times(self.h, arr))
        return {k: {"ms": arr[i].ms, "bytes": arr[i].bytes, "launches": arr[i].launches}
                for i, k in enumerate(KCLASSES)}

    # -- ABI calls -----------------------------------------------------------
    def apply_A(self, v, w=None, transpose=False):
        if w is None:
            w = self._torch.empty_like(v)
        self._check(self.lib.apply_A(self.h, self._vec(v, "v"), self._vec(w, "w"), int(bool(transpose))))
        return w

    def arnoldi(self, v0, m, want_V=True):
        V = self.empty(m + 1) if want_V else None
        H = np.zeros((m, m + 1))       # column-major (m+1) x m as rows of H^T
        beta = ctypes.c_double()
        md = ctypes.c_int()
        self._check(self.lib.arnoldi(self.h, self._vec(v0, "v0"), m,
                                     ctypes.c_void_p(V.data_ptr()) if V is not None else None,
                                     H.ctypes.data_as(ctypes.c_void_p), ctypes.byref(beta), ctypes.byref(md)))
        return V, H.T.copy(), beta.value, md.value

    def expm_phi_project(self, H, beta, tau, omegas: Optional[Sequence[float]] = None):
        H = np.asarray(H, np.float64)
        m = H.shape[1]
        Hc = np.asfortranarray(H[:m, :m])
        nf = 0 if omegas is None else len(omegas)
        om = np.ascontiguousarray(np.asarray(omegas if nf else [0.0], np.float64))
        u = np.zeros((max(1, nf), m))
        self._check(self.lib.expm_phi_project(self.h, Hc.ctypes.data_as(ctypes.c_void_p), m, m,
                                              float(beta), float(tau), _dptr(om), nf,
                                              u.ctypes.data_as(ctypes.c_void_p)))
        return u[0] if nf == 0 else u

    def stationary_solve(self, g, omegas, rtol=1e-10, max_matvecs=100000, allow_noconv=False):
        om = np.ascontiguousarray(np.asarray(omegas, np.float64))
        nf = len(om)
        zr = self._torch.zeros((nf, self.n), dtype=self.dtype, device="cuda")
        zi = self._torch.zeros((nf, self.n), dtype=self.dtype, device="cuda")
        rel = np.zeros(nf)
        mv = ctypes.c_int()
        st = self.lib.stationary_solve(self.h, self._vec(g, "g"), _dptr(om), nf, float(rtol), int(max_matvecs),
                                       ctypes.c_void_p(zr.data_ptr()), ctypes.c_void_p(zi.data_ptr()),
                                       _dptr(rel), ctypes.byref(mv))
        if not (allow_noconv and st == KX_ENOCONV):
            self._check(st)
        return zr, zi, rel, mv.value

    def expm_action(self, y0, T, rtol=1e-8, out=None):
        if out is None:
            out = self._torch.empty_like(y0)
        err = ctypes.c_double()
        self._check(self.lib.expm_action(self.h, self._vec(y0, "y0"), float(T), float(rtol),
                                         self._vec(out, "y"), ctypes.byref(err)))
        return out, err.value

    def plane_size(self, plane):
        axis = plane[0]
        p = 1
        for a in range(self.grid.dim):
            if a != axis:
                p *= self.grid.n[a]
        return (3 if self.grid.dim == 3 else 1), p

    def response_at_freqs(self, g, omegas, T, rtol=1e-8, method="split", plane=(0, 0),
                          want_plane=True, want_full=False, allow_noconv=False):
        om = np.ascontiguousarray(np.asarray(omegas, np.float64))
        nf = len(om)
        nE, npl = self.plane_size(plane)
        Ep = self._torch.empty((nf, nE, npl), dtype=self.dtype, device="cuda") if want_plane else None
        Y = self.empty(nf) if want_full else None
        inten = np.zeros(nf)
        err = np.zeros(nf)
        pl = (ctypes.c_int * 2)(int(plane[0]), int(plane[1]))
        st = self.lib.response_at_freqs(
            self.h, self._vec(g, "g"), _dptr(om), nf, float(T), float(rtol),
            METHODS[method], pl,
            ctypes.c_void_p(Ep.data_ptr()) if Ep is not None else None, _dptr(inten), _dptr(err),
            ctypes.c_void_p(Y.data_ptr()) if Y is not None else None)
        if not (allow_noconv and st == KX_ENOCONV):
            self._check(st)
        return {"E_plane": Ep, "intensity": inten, "err_est": err, "Y": Y, "status": st}

    def response_restart_dim(self, g, omegas, T, rtol=1e-8, dt_sample=0.0, max_restarts=0, plane=(0, 0),
                             want_plane=True, want_full=False, allow_noconv=False):
        """Responses by restarting in Krylov dimension (``response_restart_dim``).

        Returns E_plane, intensity, the last relative residual maxima and
        the restarts each frequency took."""
        om = np.ascontiguousarray(np.asarray(omegas, np.float64))
        nf = len(om)
        nE, npl = self.plane_size(plane)
        Ep = self._torch.empty((nf, nE, npl), dtype=self.dtype, device="cuda") if want_plane else None
        Y = self.empty(nf) if want_full else None
        inten = np.zeros(nf)
        res = np.zeros(nf)
        rst = np.zeros(nf, np.int32)
        pl = (ctypes.c_int * 2)(int(plane[0]), int(plane[1]))
        st = self.lib.response_restart_dim(
            self.h, self._vec(g, "g"), _dptr(om), nf, float(T), float(rtol), float(dt_sample), int(max_restarts),
            pl, ctypes.c_void_p(Ep.data_ptr()) if Ep is not None else None, _dptr(inten), _dptr(res),
            rst.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), ctypes.c_void_p(Y.data_ptr()) if Y is not None else None)
        if not (allow_noconv and st == KX_ENOCONV):
            self._check(st)
        return {"E_plane": Ep, "intensity": inten, "resid": res, "restarts": rst, "Y": Y, "status": st}

    def set_permittivity(self, eps_cell):
        """Replace the per-cell permittivity (numpy array or CUDA float64 tensor)."""
        torch = self._torch
        if isinstance(eps_cell, torch.Tensor) and eps_cell.is_cuda:
            e = eps_cell.detach().to(torch.float64).contiguous()
            self._check(self.lib.kx_set_permittivity(self.h, ctypes.c_void_p(e.data_ptr())))
        else:
            e = np.ascontiguousarray(np.asarray(eps_cell, np.float64).reshape(-1))
            self._check(self.lib.kx_set_permittivity(self.h, e.ctypes.data_as(ctypes.c_void_p)))

    def adjoint_response_grad(self, g, omegas, T, rtol=1e-8, plane=(0, 0)):
        """(L, dL/deps) for L = summed output-plane intensity over the frequencies.

        dL/deps is a CUDA float64 tensor with the grid's cell shape."""
        om = np.ascontiguousarray(np.asarray(omegas, np.float64))
        grad = self._torch.empty(int(np.prod(self.grid.n)), dtype=self._torch.float64, device="cuda")
        loss = ctypes.c_double()
        pl = (ctypes.c_int * 2)(int(plane[0]), int(plane[1]))
        self._check(self.lib.adjoint_response_grad(self.h, self._vec(g, "g"), _dptr(om), len(om), float(T),
                                                   float(rtol), pl, ctypes.c_void_p(grad.data_ptr()),
                                                   ctypes.byref(loss)))
        return loss.value, grad.reshape(tuple(reversed(self.grid.n)))


def intensity_loss(ctx, eps_cell, g, omegas, T, rtol=1e-8, plane=(0, 0)):
    """Differentiable summed output-plane intensity L(eps) (torch scalar).

    Forward and gradient both come from ``adjoint_response_grad``; the
    context's permittivity is replaced by ``eps_cell`` first."""
    import torch

    class _IntensityLoss(torch.autograd.Function):
        @staticmethod
        def forward(fctx, eps):
            ctx.set_permittivity(eps)
            loss, grad = ctx.adjoint_response_grad(g, omegas, T, rtol, plane)
            fctx.save_for_backward(grad)
            return torch.tensor(loss, dtype=torch.float64, device=eps.device)

        @staticmethod
        def backward(fctx, gout):
            (grad,) = fctx.saved_tensors
            return gout * grad.to(gout.device)

    return _IntensityLoss.apply(eps_cell)


def response_multi(ctxs, gs, omegas, T, rtol=1e-8, method="plain", planes=None, nthreads=8):
    """Independent problems concurrently (``response_at_freqs_multi``).

    ctxs: Contexts (distinct non-default streams); gs: their source tensors;
    omegas: (nctx, nfreq) array; planes: (nctx, 2).  Returns (intensity,
    err_est), each (nctx, nfreq)."""
    lib = load_library()
    n = len(ctxs)
    om = np.ascontiguousarray(np.asarray(omegas, np.float64).reshape(n, -1))
    nf = om.shape[1]
    pl = np.ascontiguousarray(np.asarray(planes, np.int32).reshape(n, 2))
    hs = (ctypes.c_void_p * n)(*[c.h for c in ctxs])
    gp = (ctypes.c_void_p * n)(*[c._vec(g, "g").value for c, g in zip(ctxs, gs)])
    inten = np.zeros((n, nf))
    err = np.zeros((n, nf))
    st = lib.response_at_freqs_multi(hs, n, gp, _dptr(om), nf, float(T), float(rtol),
                                     METHODS[method],
                                     pl.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dptr(inten), _dptr(err),
                                     int(nthreads))
    if st != KX_OK:
        raise KxError(st, lib.kx_last_error(None).decode())
    return inten, err


class Batch:
    """Many independent problems solved together by restart in Krylov
    dimension (``kx_batch_create`` / ``response_restart_dim_batch``): one
    launch per Arnoldi phase serves every problem.  ``ctxs``: 3D FP32
    Contexts (n[0] a multiple of 4, batch >= 2, rst_samples > 0, one
    krylov_dim); they must outlive the Batch.  ``stream``: a torch CUDA
    stream, or "own"."""

    def __init__(self, ctxs, stream="own"):
        import torch
        self.lib = load_library()
        self.ctxs = list(ctxs)
        own = isinstance(stream, str) and stream == "own"
        sarg = ctypes.c_void_p(-1) if own else ctypes.c_void_p(stream.cuda_stream)
        hs = (ctypes.c_void_p * len(self.ctxs))(*[c.h for c in self.ctxs])
        h = ctypes.c_void_p()
        st = self.lib.kx_batch_create(hs, len(self.ctxs), sarg, ctypes.byref(h))
        if st != KX_OK:
            raise KxError(st, self.lib.kx_batch_last_error(None).decode())
        self.h = h

    def set_timing(self, on: bool):
        self.lib.kx_batch_set_timing(self.h, int(bool(on)))

    def info(self):
        i = BatchInfo()
        self.lib.kx_batch_get_info(self.h, ctypes.byref(i))
        return {k: getattr(i, k) for k, _ in BatchInfo._fields_}

    def response(self, gs, omegas, T, rtol=1e-7, max_restarts=0, planes=None, allow_noconv=False):
        """(intensity, resid, restarts), each (nproblems, nfreq)."""
        n = len(self.ctxs)
        om = np.ascontiguousarray(np.asarray(omegas, np.float64).reshape(n, -1))
        nf = om.shape[1]
        pl = np.ascontiguousarray(np.asarray(planes, np.int32).reshape(n, 2))
        gp = (ctypes.c_void_p * n)(*[c._vec(g, "g").value for c, g in zip(self.ctxs, gs)])
        inten = np.zeros((n, nf))
        res = np.zeros((n, nf))
        rst = np.zeros((n, nf), np.int32)
        st = self.lib.response_restart_dim_batch(self.h, gp, _dptr(om), nf, float(T), float(rtol), int(max_restarts),
                                                 pl.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _dptr(inten),
                                                 _dptr(res), rst.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
        if not (allow_noconv and st == KX_ENOCONV) and st != KX_OK:
            raise KxError(st, self.lib.kx_batch_last_error(self.h).decode())
        return inten, res, rst

    def close(self):
        if getattr(self, "h", None):
            self.lib.kx_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

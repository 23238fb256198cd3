"""Thin ctypes binding of libosvmbe (C ABI in include/osvmbe.h).  Argument marshalling only: every step of the
method runs in the library's CUDA kernels.  PyTorch provides device memory and the stream.

Raises RuntimeError when the library is missing or the device is not a CUDA GPU: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libosvmbe.so")

OSV_OK, OSV_ERR_INVALID, OSV_ERR_NOCONV, OSV_ERR_OOM, OSV_ERR_CUDA, OSV_ERR_TIMEOUT, OSV_ERR_NUMERIC = \
    0, -1, -2, -3, -4, -5, -6
OSV_FP64, OSV_MIXED_TF32X3, OSV_MIXED_BF16X4 = 0, 1, 2

EXPORTS = ["osv_create", "osv_destroy", "osv_last_error", "clusters_build", "osv_build", "cluster_residual_solve",
           "mbe3_combine", "energy", "gradient_backward", "osv_cluster_count", "osv_cluster_info",
           "osv_eigenvalues", "osv_syev_batched", "osv_profile_enable", "osv_profile_read",
           "osv_residual_flops", "osv_kernel_launches", "osv_syev_batched_noalloc", "osv_adjoint_flops",
           "osv_solve_counts", "osv_residual_work", "osv_set_wait_budget",
           "osv_pair_amplitudes", "osv_overlap_metric", "clusters_build_osv",
           "posterior_correction", "weak_pairs_energy", "osv_autotune", "osv_autotune_report",
           "osv_graph_capture", "osv_graph_launch", "osv_graph_kernels", "osv_set_tridiag_variant"]


class OsvParams(ctypes.Structure):
    _fields_ = [("l_osv", ctypes.c_double), ("n_osv_max", ctypes.c_int), ("n_osv_fixed", ctypes.c_int),
                ("r2b", ctypes.c_double), ("r3b", ctypes.c_double), ("mbe_order", ctypes.c_int),
                ("tau_red", ctypes.c_double), ("tol", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("precision", ctypes.c_int)]


class OsvProblem(ctypes.Structure):
    _fields_ = [("n_occ", ctypes.c_int), ("n_vir", ctypes.c_int), ("n_aux", ctypes.c_int),
                ("centres", ctypes.c_void_p), ("aux_ptr", ctypes.c_void_p), ("aux_idx", ctypes.c_void_p),
                ("f_occ", ctypes.c_void_p), ("eps_vir", ctypes.c_void_p), ("B", ctypes.c_void_p),
                ("B_dtype", ctypes.c_int)]


_lib = None


def load(path=LIB_PATH):
    """Load libosvmbe.so (built in-tree by paper_2106_06149_gb300.build) and declare its signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2106_06149_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P, I, D, V = ctypes.POINTER, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
    sig = {
        "osv_create": ([P(V), V], I),
        "osv_destroy": ([V], I),
        "osv_last_error": ([V], ctypes.c_char_p),
        "clusters_build": ([V, P(OsvProblem), P(OsvParams), V], I),
        "osv_build": ([V, P(OsvProblem), P(OsvParams), V], I),
        "cluster_residual_solve": ([V, V, V], I),
        "mbe3_combine": ([V], I),
        "energy": ([V, P(D), V], I),
        "gradient_backward": ([V, D, V, V], I),
        "osv_cluster_count": ([V, P(I)], I),
        "osv_cluster_info": ([V, V, V, V, V], I),
        "osv_eigenvalues": ([V, I, V], I),
        "osv_syev_batched": ([V, I, I, V, V, V], I),
        "osv_profile_enable": ([V, I], I),
        "osv_profile_read": ([V, I, V, V, V, P(I)], I),
        "osv_residual_flops": ([V, P(D)], I),
        "osv_kernel_launches": ([P(ctypes.c_longlong)], I),
        "osv_syev_batched_noalloc": ([V, I, I, V, V, V], I),
        "osv_adjoint_flops": ([V, P(D)], I),
        "osv_solve_counts": ([V, P(ctypes.c_longlong), P(ctypes.c_longlong), P(I)], I),
        "osv_residual_work": ([V, P(D), P(D)], I),
        "osv_set_wait_budget": ([V, ctypes.c_longlong], I),
        "osv_pair_amplitudes": ([V, I, I, V], I),
        "osv_overlap_metric": ([V, P(OsvProblem), P(OsvParams), V], I),
        "clusters_build_osv": ([V, P(OsvProblem), P(OsvParams), V, D, D, V], I),
        "posterior_correction": ([V, P(D), P(D), P(D)], I),
        "weak_pairs_energy": ([V, V, D, D, P(D), P(I)], I),
        "osv_autotune": ([V, I], I),
        "osv_autotune_report": ([V, V, I, P(I)], I),
        "osv_graph_capture": ([V, P(OsvProblem), P(OsvParams), D, V, V], I),
        "osv_graph_launch": ([V, P(D), P(D)], I),
        "osv_graph_kernels": ([V, P(ctypes.c_longlong)], I),
        "osv_set_tridiag_variant": ([V, I], I),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


class OsvError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"libosvmbe status {status}: {msg}")
        self.status = status


def _check(status, ctx=None):
    if status != OSV_OK:
        msg = load().osv_last_error(ctx).decode()
        raise OsvError(status, msg)


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data if isinstance(a, np.ndarray) else a.data_ptr())


def _stream_handle(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def params_struct(params):
    d = params if isinstance(params, dict) else params.as_dict()
    return OsvParams(l_osv=d["l_osv"], n_osv_max=d["n_osv_max"], n_osv_fixed=d["n_osv_fixed"], r2b=d["r2b"],
                     r3b=d["r3b"], mbe_order=d["mbe_order"], tau_red=d["tau_red"], tol=d["tol"],
                     max_iter=d["max_iter"], precision=d["precision"])


class DeviceProblem:
    """A problem with its DF tensor, occupied Fock matrix and virtual energies resident on the GPU."""

    def __init__(self, centres, aux_ptr, aux_idx, f_occ, eps_vir, B, n_aux):
        if not torch.cuda.is_available():
            raise RuntimeError("libosvmbe needs a CUDA device")
        self.centres = np.ascontiguousarray(centres, dtype=np.float64)
        self.aux_ptr = np.ascontiguousarray(aux_ptr, dtype=np.int64)
        self.aux_idx = np.ascontiguousarray(aux_idx, dtype=np.int32)
        self.f_occ = f_occ
        self.eps_vir = eps_vir
        self.B = B
        self.n_aux = int(n_aux)
        for t in (f_occ, eps_vir, B):
            if not (t.is_cuda and t.is_contiguous()):
                raise ValueError("f_occ, eps_vir and B must be contiguous CUDA tensors")
        if f_occ.dtype != torch.float64 or eps_vir.dtype != torch.float64:
            raise ValueError("f_occ and eps_vir must be float64")
        if B.dtype not in (torch.float64, torch.float32):
            raise ValueError("B must be float64 or float32")

    @classmethod
    def from_host(cls, p, device="cuda", pin=False):
        """Copy a synth.Problem (numpy arrays) to the device."""
        def dev(a, dt):
            t = torch.from_numpy(np.ascontiguousarray(a)).to(dt)
            if pin:
                t = t.pin_memory()
            return t.to(device, non_blocking=pin)
        Bdt = torch.float32 if p.B.dtype == np.float32 else torch.float64
        return cls(p.centres, p.aux_ptr, p.aux_idx, dev(p.f_occ, torch.float64), dev(p.eps_vir, torch.float64),
                   dev(p.B, Bdt), p.aux_centres.shape[0])

    @property
    def n_occ(self):
        return self.centres.shape[0]

    @property
    def n_vir(self):
        return self.eps_vir.shape[0]

    def struct(self, B=None, f_occ=None):
        B = self.B if B is None else B
        f = self.f_occ if f_occ is None else f_occ
        return OsvProblem(n_occ=self.n_occ, n_vir=self.n_vir, n_aux=self.n_aux, centres=_ptr(self.centres),
                          aux_ptr=_ptr(self.aux_ptr), aux_idx=_ptr(self.aux_idx), f_occ=_ptr(f),
                          eps_vir=_ptr(self.eps_vir), B=_ptr(B), B_dtype=0 if B.dtype == torch.float64 else 1)


class Context:
    """One libosvmbe context (osv_ctx) bound to a CUDA stream."""

    def __init__(self, stream=None):
        lib = load()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        _check(lib.osv_create(ctypes.byref(h), _stream_handle(self.stream)))
        self.h = h
        self._keep = None

    def close(self):
        if getattr(self, "h", None):
            load().osv_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- the five calls of the C ABI (same names)
    def clusters_build(self, prob: DeviceProblem, params):
        self._prm = params_struct(params)
        ps = prob.struct()
        n = (ctypes.c_int * 3)()
        _check(load().clusters_build(self.h, ctypes.byref(ps), ctypes.byref(self._prm), n), self.h)
        return [n[0], n[1], n[2]]

    def osv_overlap_metric(self, prob: DeviceProblem, params):
        """OSV-overlap metric s2b (n_occ x n_occ) of Eq. 2bscreen from the OSVs of every LMO."""
        self._prm = params_struct(params)
        ps = prob.struct()
        out = np.zeros((prob.n_occ, prob.n_occ), np.float64)
        _check(load().osv_overlap_metric(self.h, ctypes.byref(ps), ctypes.byref(self._prm), _ptr(out)), self.h)
        return out

    def clusters_build_osv(self, prob: DeviceProblem, params, s2b, l2b, l3b):
        """clusters_build with the 2b/3b selection of Eqs. 2bscreen and 3bscreen on the metric s2b."""
        self._prm = params_struct(params)
        ps = prob.struct()
        s = np.ascontiguousarray(s2b, dtype=np.float64)
        n = (ctypes.c_int * 3)()
        _check(load().clusters_build_osv(self.h, ctypes.byref(ps), ctypes.byref(self._prm), _ptr(s), float(l2b),
                                         float(l3b), n), self.h)
        return [n[0], n[1], n[2]]

    def osv_build(self, prob: DeviceProblem, params=None, want_counts=False, B=None, f_occ=None):
        if params is not None:
            self._prm = params_struct(params)
        ps = prob.struct(B=B, f_occ=f_occ)
        self._keep = (prob, B, f_occ)
        out = np.zeros(prob.n_occ, dtype=np.int32) if want_counts else None
        _check(load().osv_build(self.h, ctypes.byref(ps), ctypes.byref(self._prm),
                                _ptr(out) if want_counts else None), self.h)
        return out

    def cluster_residual_solve(self, want_iters=False, status=None):
        it = ctypes.c_int(0)
        _check(load().cluster_residual_solve(self.h, ctypes.byref(it) if want_iters else None,
                                             _ptr(status) if status is not None else None), self.h)
        return it.value if want_iters else None

    def mbe3_combine(self):
        _check(load().mbe3_combine(self.h), self.h)

    def energy(self):
        e = ctypes.c_double()
        el = ctypes.c_double()
        _check(load().energy(self.h, ctypes.byref(e), ctypes.byref(el)), self.h)
        return e.value, el.value

    def weak_pairs_energy(self, s2b, l2b, l_discard=1e-7):
        """One-block energies of the weak pairs (Sec. 2.2.2): (E_weak, number of weak pairs)."""
        s = np.ascontiguousarray(s2b, dtype=np.float64)
        e, n = ctypes.c_double(), ctypes.c_int()
        _check(load().weak_pairs_energy(self.h, _ptr(s), float(l2b), float(l_discard), ctypes.byref(e),
                                        ctypes.byref(n)), self.h)
        return e.value, n.value

    def posterior_correction(self):
        """One-step posterior correction (Sec. 3): dict(E_global, E_corrected, dR_max)."""
        eg, ec, r = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(load().posterior_correction(self.h, ctypes.byref(eg), ctypes.byref(ec), ctypes.byref(r)), self.h)
        return dict(E_global=eg.value, E_corrected=ec.value, dR_max=r.value)

    def gradient_backward(self, scale, dB=None, dF=None):
        _check(load().gradient_backward(self.h, float(scale), _ptr(dB) if dB is not None else None,
                                        _ptr(dF) if dF is not None else None), self.h)

    def graph_capture(self, prob: DeviceProblem, params=None, scale=1.0, dB=None, dF=None, B=None, f_occ=None):
        """Run one eager step, then record the whole step (build, solves, combination, energy and, with dB or dF,
        the adjoint into those buffers, which each replay overwrites) as a CUDA graph.  The graph keeps the device
        addresses of the problem arrays and of dB/dF: update their values in place between graph_launch calls."""
        if params is not None:
            self._prm = params_struct(params)
        ps = prob.struct(B=B, f_occ=f_occ)
        self._keep = (prob, B, f_occ)
        self._graph_keep = (prob, B, f_occ, dB, dF)
        _check(load().osv_graph_capture(self.h, ctypes.byref(ps), ctypes.byref(self._prm), float(scale),
                                        _ptr(dB) if dB is not None else None, _ptr(dF) if dF is not None else None),
               self.h)

    def graph_launch(self):
        """Replay the recorded step; returns (E, E_linear)."""
        E, El = ctypes.c_double(), ctypes.c_double()
        _check(load().osv_graph_launch(self.h, ctypes.byref(E), ctypes.byref(El)), self.h)
        return E.value, El.value

    def graph_kernels(self):
        n = ctypes.c_longlong()
        _check(load().osv_graph_kernels(self.h, ctypes.byref(n)), self.h)
        return n.value

    def set_tridiag_variant(self, variant):
        """Fix the FP32 tridiagonalisation's launch shape for later plans (0-4), or -1 to tune it."""
        _check(load().osv_set_tridiag_variant(self.h, int(variant)), self.h)

    def autotune(self, on=True):
        """Plan-time autotuning of launch shapes (mixed precision); on by default."""
        _check(load().osv_autotune(self.h, 1 if on else 0), self.h)

    def autotune_report(self):
        """The last plan's tuned launch shapes (dict; empty when nothing was tuned)."""
        import json
        n = ctypes.c_int()
        _check(load().osv_autotune_report(self.h, None, 0, ctypes.byref(n)), self.h)
        buf = ctypes.create_string_buffer(max(n.value, 1))
        _check(load().osv_autotune_report(self.h, buf, n.value, ctypes.byref(n)), self.h)
        return json.loads(buf.value.decode()) if buf.value else {}

    def set_wait_budget(self, cycles):
        """Bound (SM clock cycles) of the tensor-core kernels' pipeline waits; <= 0 restores the default."""
        _check(load().osv_set_wait_budget(self.h, int(cycles)), self.h)

    # --- diagnostics
    def cluster_info(self):
        n = ctypes.c_int()
        _check(load().osv_cluster_count(self.h, ctypes.byref(n)), self.h)
        mem = np.zeros((n.value, 3), np.int32)
        w = np.zeros(n.value, np.int32)
        e = np.zeros(n.value, np.float64)
        it = np.zeros(n.value, np.int32)
        _check(load().osv_cluster_info(self.h, _ptr(mem), _ptr(w), _ptr(e), _ptr(it)), self.h)
        return mem, w, e, it

    def profile(self, on=True):
        _check(load().osv_profile_enable(self.h, 1 if on else 0), self.h)

    def profile_read(self):
        """{stage: (total_ms, records)} of the stages recorded since profiling was enabled."""
        n = ctypes.c_int()
        _check(load().osv_profile_read(self.h, 0, None, None, None, ctypes.byref(n)), self.h)
        names = ctypes.create_string_buffer(32 * max(n.value, 1))
        ms = np.zeros(max(n.value, 1), np.float64)
        calls = np.zeros(max(n.value, 1), np.int32)
        _check(load().osv_profile_read(self.h, n.value, names, _ptr(ms), _ptr(calls), ctypes.byref(n)), self.h)
        raw = names.raw
        return {raw[32 * q:32 * q + 32].split(b"\0")[0].decode(): (float(ms[q]), int(calls[q]))
                for q in range(n.value)}

    def residual_flops(self):
        f = ctypes.c_double()
        _check(load().osv_residual_flops(self.h, ctypes.byref(f)), self.h)
        return f.value

    def adjoint_flops(self):
        f = ctypes.c_double()
        _check(load().osv_adjoint_flops(self.h, ctypes.byref(f)), self.h)
        return f.value

    def solve_counts(self):
        """(FP32 Jacobi updates, FP64-accurate residual evaluations, unconverged clusters) of the last solve."""
        u, f, bad = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_int()
        _check(load().osv_solve_counts(self.h, ctypes.byref(u), ctypes.byref(f), ctypes.byref(bad)), self.h)
        return u.value, f.value, bad.value

    def residual_work(self):
        """(FLOPs of FP32 residual evaluations, FLOPs of FP64-accurate evaluations) of the last solve."""
        f32, f64 = ctypes.c_double(), ctypes.c_double()
        _check(load().osv_residual_work(self.h, ctypes.byref(f32), ctypes.byref(f64)), self.h)
        return f32.value, f64.value

    def pair_amplitudes(self, i, j, n_vir):
        """Collective amplitudes t_ij of the ordered pair (i, j) in the canonical virtual space (n_vir x n_vir)."""
        out = np.zeros((n_vir, n_vir), np.float64)
        _check(load().osv_pair_amplitudes(self.h, int(i), int(j), _ptr(out)), self.h)
        return out

    def eigenvalues(self, k, n_vir):
        out = np.zeros(n_vir, np.float64)
        _check(load().osv_eigenvalues(self.h, int(k), _ptr(out)), self.h)
        return out


def syev_batched(A: torch.Tensor, stream=None):
    """Eigen-decompose a batch of symmetric (batch, n, n) float64 CUDA matrices: (w decreasing, Zt rows)."""
    A = A.contiguous()
    b, n, _ = A.shape
    w = torch.empty(b, n, dtype=torch.float64, device=A.device)
    Zt = torch.empty(b, n, n, dtype=torch.float64, device=A.device)
    _check(load().osv_syev_batched(_ptr(A), n, b, _ptr(w), _ptr(Zt), _stream_handle(stream)))
    return w, Zt


def kernel_launches():
    """Kernels the library has launched in this process (osv_kernel_launches)."""
    n = ctypes.c_longlong()
    _check(load().osv_kernel_launches(ctypes.byref(n)))
    return n.value


def run_energy(ctx: Context, prob: DeviceProblem, params, B=None, f_occ=None):
    """osv_build -> cluster_residual_solve -> mbe3_combine -> energy.  Returns (E, E_linear)."""
    ctx.osv_build(prob, params, B=B, f_occ=f_occ)
    ctx.cluster_residual_solve()
    ctx.mbe3_combine()
    return ctx.energy()


class Energy(torch.autograd.Function):
    """E = MBE(3)-OSV-MP2 energy of (B, F_occ); backward is the library's adjoint (gradient_backward)."""

    @staticmethod
    def forward(fctx, B, f_occ, ctx: Context, prob: DeviceProblem, params):
        B = B.contiguous()
        f_occ = f_occ.contiguous()
        E, _ = run_energy(ctx, prob, params, B=B, f_occ=f_occ)
        fctx.lib_ctx = ctx
        fctx.save_for_backward(B, f_occ)
        return torch.tensor(E, dtype=torch.float64, device=B.device)

    @staticmethod
    def backward(fctx, gE):
        B, f_occ = fctx.saved_tensors
        dB = torch.zeros_like(B) if fctx.needs_input_grad[0] else None
        dF = torch.zeros_like(f_occ) if fctx.needs_input_grad[1] else None
        fctx.lib_ctx.gradient_backward(float(gE), dB, dF)
        return dB, dF, None, None, None

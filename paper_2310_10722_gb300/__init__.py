"""GB300-native tensor-network coset decoder (arXiv 2310.10722), Python binding.

Thin argument marshalling over the C ABI of libtd.so (include/td.h): every step of the
decoding path runs in the library's CUDA kernels.  PyTorch supplies device memory and
streams.  Importing this package does not load the library; the first Network does, and
raises if libtd.so has not been built (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from ._lib import TD_FP32, TD_FP64, TD_TC, TDError, check

__all__ = ["Network", "GenNetwork", "TDError", "TD_FP64", "TD_FP32", "TD_TC", "load_library"]


def load_library():
    return _lib.load()


def _i32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


class Network:
    """A built decoding network (td_build_network) and its device workspace.

    H and l are given in CSR by rows (detectors x mechanisms, observables x mechanisms),
    `p` the mechanism rates, `det_xyt` the (x, y, t) of every detector.
    """

    def __init__(self, H_indptr, H_indices, L_indptr, L_indices, p, det_xyt, *, n_mech=None,
                 chi=8, chi_mps=16, precision=TD_FP64, svd_cutoff=1e-12, multiplet_rtol=1e-8,
                 gram_cutoff=None, mem_budget=0, max_wave=0, ckpt_stride=0):
        lib = _lib.load()
        self._lib = lib
        self._keep = [_i32(H_indptr), _i32(H_indices), _i32(L_indptr), _i32(L_indices),
                      np.ascontiguousarray(np.asarray(p, dtype=np.float64)), _i32(det_xyt).reshape(-1)]
        hip, hix, lip, lix, pp, xyt = self._keep
        n_det = len(hip) - 1
        n_obs = len(lip) - 1
        n_mech = len(pp) if n_mech is None else n_mech
        P = lambda a, t: a.ctypes.data_as(C.POINTER(t))
        dem = _lib.td_dem(n_det, n_mech, n_obs, P(hip, C.c_int32), P(hix, C.c_int32), P(lip, C.c_int32),
                          P(lix, C.c_int32), P(pp, C.c_double))
        lay = _lib.td_layout(P(xyt, C.c_int32))
        opt = _lib.td_options()
        lib.td_default_options(C.byref(opt))
        opt.chi, opt.chi_mps, opt.precision = chi, chi_mps, precision
        opt.svd_cutoff, opt.multiplet_rtol = svd_cutoff, multiplet_rtol
        if gram_cutoff is not None:
            opt.gram_cutoff = gram_cutoff
        if mem_budget:
            opt.mem_budget = mem_budget
        opt.max_wave = max_wave
        opt.ckpt_stride = ckpt_stride
        h = C.c_void_p()
        check(lib.td_build_network(C.byref(dem), C.byref(lay), C.byref(opt), C.byref(h)))
        self._h = h
        self.n_det, self.n_mech, self.n_obs = n_det, n_mech, n_obs
        self.n_class = 1 << n_obs

    @classmethod
    def from_dem(cls, dem, **kw):
        """Build from any object with H_csr(), L_csr(), p, det_xyt (e.g. td_inputs.DEM)."""
        hip, hix = dem.H_csr()
        lip, lix = dem.L_csr()
        return cls(hip, hix, lip, lix, dem.p, dem.det_xyt, n_mech=dem.n_mech, **kw)

    def info(self) -> dict:
        inf = _lib.td_network_info()
        check(self._lib.td_network_get_info(self._h, C.byref(inf)))
        return {k: getattr(inf, k) for k, _ in inf._fields_}

    def check(self, stream=None):
        """td_network_check: synchronise the stream and raise if a kernel recorded an error
        status (TD_ERR_TIMEOUT: a bounded device wait gave up) since the last check."""
        check(self._lib.td_network_check(self._h, self._stream(stream)))

    @staticmethod
    def _stream(stream):
        import torch
        s = stream if stream is not None else torch.cuda.current_stream()
        return C.c_void_p(s.cuda_stream)

    def _check_det(self, det):
        import torch
        if not (isinstance(det, torch.Tensor) and det.is_cuda and det.dtype == torch.uint8 and det.dim() == 2
                and det.shape[1] == self.n_det and det.is_contiguous()):
            raise ValueError(f"det must be a contiguous CUDA uint8 tensor [B, {self.n_det}]")

    def coset_logprob(self, det, out=None, stream=None):
        """log p_{m,L} for every shot: CUDA float64 [B, 2^n_obs]."""
        import torch
        self._check_det(det)
        B = det.shape[0]
        if out is None:
            out = torch.empty((B, self.n_class), dtype=torch.float64, device=det.device)
        check(self._lib.td_coset_logprob(self._h, C.c_void_p(det.data_ptr()), B, C.c_void_p(out.data_ptr()),
                                         self._stream(stream)))
        return out

    def coset_logprob_stats(self, det, stream=None):
        """(log p_{m,L} [B, 2], truncation statistics [B, 4]) on the device: per shot the
        largest and the summed discarded fraction of the simple-update truncations, then of
        the final contraction's cuts (td_coset_logprob_stats)."""
        import torch
        self._check_det(det)
        B = det.shape[0]
        out = torch.empty((B, self.n_class), dtype=torch.float64, device=det.device)
        stats = torch.empty((B, 4), dtype=torch.float64, device=det.device)
        check(self._lib.td_coset_logprob_stats(self._h, C.c_void_p(det.data_ptr()), B, C.c_void_p(out.data_ptr()),
                                               C.c_void_p(stats.data_ptr()), self._stream(stream)))
        return out, stats

    def decode(self, det, stream=None):
        """(decision int32 [B], margin float64 [B]) on the device."""
        import torch
        self._check_det(det)
        B = det.shape[0]
        dec = torch.empty(B, dtype=torch.int32, device=det.device)
        mar = torch.empty(B, dtype=torch.float64, device=det.device)
        check(self._lib.td_decode(self._h, C.c_void_p(det.data_ptr()), B, C.c_void_p(dec.data_ptr()),
                                  C.c_void_p(mar.data_ptr()), self._stream(stream)))
        return dec, mar

    def coset_logprob_host(self, det, out=None, stream=None):
        """Host-buffer variant: det uint8 [B, n_det] (numpy or CPU tensor, ideally pinned);
        returns float64 [B, 2^n_obs] in host memory.  Synchronises the stream."""
        import torch
        if isinstance(det, np.ndarray):
            det = torch.from_numpy(np.ascontiguousarray(det, dtype=np.uint8))
        if det.is_cuda or det.dtype != torch.uint8 or det.dim() != 2 or det.shape[1] != self.n_det:
            raise ValueError(f"det must be a host uint8 tensor [B, {self.n_det}]")
        det = det.contiguous()
        B = det.shape[0]
        if out is None:
            out = torch.empty((B, self.n_class), dtype=torch.float64, pin_memory=det.is_pinned())
        check(self._lib.td_coset_logprob_host(self._h, C.c_void_p(det.data_ptr()), B,
                                              C.c_void_p(out.data_ptr()), self._stream(stream)))
        return out

    def grad_logprob(self, det, p=None, stream=None, method="reverse"):
        """(log P [B], d mean_b log P / d p [n_mech]) with P(m) = sum_L p_{m,L}, on det's
        device.  p: float64 rates on the device (None: the current rates); a given p
        becomes the network's rates for later calls too.  method "reverse": the reverse
        sweep (td_grad_logprob); "forced": the affine identity by forced decodes
        (td_grad_logprob_forced)."""
        import torch
        self._check_det(det)
        B = det.shape[0]
        logP = torch.empty(B, dtype=torch.float64, device=det.device)
        grad = torch.empty(self.n_mech, dtype=torch.float64, device=det.device)
        if p is not None:
            if p.dtype != torch.float64 or p.device != det.device or p.numel() != self.n_mech:
                raise ValueError("p must be float64 [n_mech] on the detector buffer's device")
            p = p.contiguous()
        pp = C.c_void_p(p.data_ptr()) if p is not None else None
        fn = {"reverse": self._lib.td_grad_logprob, "forced": self._lib.td_grad_logprob_forced}[method]
        check(fn(self._h, C.c_void_p(det.data_ptr()), B, pp, C.c_void_p(logP.data_ptr()),
                 C.c_void_p(grad.data_ptr()), self._stream(stream)))
        return logP, grad

    def set_schedule(self, final_threads: int, chunk_rows: int, final_smem: bool = True):
        """Launch schedule: k_final block size (256/512/1024) and work region in shared memory
        (when it fits) or global memory, Gram/update rows per job (512..4096)."""
        check(self._lib.td_network_set_schedule(self._h, int(final_threads), int(bool(final_smem)), int(chunk_rows)))

    def tune(self, det, stream=None) -> dict:
        """Autotune the launch schedule on decodes of det's first min(B, wave) shots; keeps
        and returns the fastest {final_threads, chunk_rows, ms}."""
        self._check_det(det)
        th, sm, cr, ms = C.c_int32(), C.c_int32(), C.c_int32(), C.c_double()
        check(self._lib.td_network_tune(self._h, C.c_void_p(det.data_ptr()), det.shape[0], C.byref(th),
                                        C.byref(sm), C.byref(cr), C.byref(ms), self._stream(stream)))
        return {"final_threads": th.value, "final_smem": bool(sm.value), "chunk_rows": cr.value, "ms": ms.value}

    def debug_sweep(self, det, n_gates, stream=None):
        """Bond weights [B, n_bonds, chi] and log-scale slots after the first n_gates gates
        (rounded up to a whole gate round); returns (lam, logacc, applied)."""
        import torch
        self._check_det(det)
        inf = self.info()
        B = min(det.shape[0], inf["wave"])
        lam = torch.zeros((B, inf["n_bonds"], inf["chi"]), dtype=torch.float64, device=det.device)
        la = torch.zeros((B, inf["n_sites"] + inf["n_bonds"] + 1), dtype=torch.float64, device=det.device)
        applied = C.c_int32()
        check(self._lib.td_debug_sweep(self._h, C.c_void_p(det.data_ptr()), B, n_gates, C.c_void_p(lam.data_ptr()),
                                       C.c_void_p(la.data_ptr()), C.byref(applied), self._stream(stream)))
        return lam, la, applied.value

    def profile(self, enable: bool):
        """Start (True) or stop (False) per-launch CUDA-event timing; returns the totals
        recorded so far as {kernel class: (ms, launches)}."""
        ms = (C.c_double * 8)()
        n = (C.c_int64 * 8)()
        check(self._lib.td_network_profile(self._h, int(enable), C.cast(ms, C.c_void_p), C.cast(n, C.c_void_p)))
        return {k: (ms[i], n[i]) for i, k in enumerate(_lib.KERNEL_CLASSES)}

    def work(self) -> dict:
        """Algorithmic work per shot per kernel class: {class: (bytes, flops, fp64_flops)}."""
        b, f, f64 = (C.c_double * 8)(), (C.c_double * 8)(), (C.c_double * 8)()
        check(self._lib.td_network_get_work(self._h, C.cast(b, C.c_void_p), C.cast(f, C.c_void_p),
                                            C.cast(f64, C.c_void_p)))
        return {k: (b[i], f[i], f64[i]) for i, k in enumerate(_lib.KERNEL_CLASSES)}

    def close(self):
        if getattr(self, "_h", None):
            self._lib.td_free_network(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class GenNetwork(Network):
    """A generator network (td_build_gen_network, Sec. 3.2): a CSS sector decoded in the
    generator picture, e.g. the loop sector of the 3D surface code (Sec. 5.2).

    qubit_gens [n_qubits][2]: the generators flipping each qubit (second -1 for a dangling
    edge); p the flip rates; gen_xyt [n_gen][3]; the checks H in CSR by rows; xbar, zbar
    the qubits of the flipped-type logical and of its conjugate (the class of an error).
    """

    def __init__(self, qubit_gens, p, gen_xyt, check_indptr, check_indices, xbar, zbar, *, chi=8, chi_mps=16,
                 precision=TD_FP64, svd_cutoff=1e-12, multiplet_rtol=1e-8, gram_cutoff=None, mem_budget=0,
                 max_wave=0):
        lib = _lib.load()
        self._lib = lib
        qg = _i32(qubit_gens).reshape(-1)
        self._keep = [qg, np.ascontiguousarray(np.asarray(p, dtype=np.float64)), _i32(gen_xyt).reshape(-1),
                      _i32(check_indptr), _i32(check_indices), _i32(xbar), _i32(zbar)]
        qg, pp, xyt, cip, cix, xb, zb = self._keep
        P = lambda a, t: a.ctypes.data_as(C.POINTER(t))
        g = _lib.td_gen(len(xyt) // 3, len(qg) // 2, len(cip) - 1, P(qg, C.c_int32), P(pp, C.c_double),
                        P(xyt, C.c_int32), P(cip, C.c_int32), P(cix, C.c_int32), len(xb), P(xb, C.c_int32),
                        len(zb), P(zb, C.c_int32))
        opt = _lib.td_options()
        lib.td_default_options(C.byref(opt))
        opt.chi, opt.chi_mps, opt.precision = chi, chi_mps, precision
        opt.svd_cutoff, opt.multiplet_rtol = svd_cutoff, multiplet_rtol
        if gram_cutoff is not None:
            opt.gram_cutoff = gram_cutoff
        if mem_budget:
            opt.mem_budget = mem_budget
        opt.max_wave = max_wave
        h = C.c_void_p()
        check(lib.td_build_gen_network(C.byref(g), C.byref(opt), C.byref(h)))
        self._h = h
        self.n_checks = len(cip) - 1
        self.n_qubits = len(qg) // 2
        self.n_det, self.n_mech, self.n_obs, self.n_class = self.n_checks, self.n_qubits, 1, 2

    @classmethod
    def from_problem(cls, gp, **kw):
        """Build from a td_inputs.GenProblem (edges, p, gen_xyt, xbar, zbar, face_dem)."""
        qg = np.array([list(e) + [-1] * (2 - len(e)) for e in gp.edges], dtype=np.int32)
        hip, hix = gp.face_dem.H_csr()
        return cls(qg, gp.p, gp.gen_xyt, hip, hix, list(gp.xbar), list(gp.zbar), **kw)

    def coset_logprob(self, syn, out=None, stream=None):
        """log p_{m,L} for every shot: CUDA float64 [B, 2] (syn: CUDA uint8 [B, n_checks])."""
        import torch
        self._check_det(syn)
        B = syn.shape[0]
        if out is None:
            out = torch.empty((B, 2), dtype=torch.float64, device=syn.device)
        check(self._lib.td_gen_coset_logprob(self._h, C.c_void_p(syn.data_ptr()), B, C.c_void_p(out.data_ptr()),
                                             self._stream(stream)))
        return out

    def decode(self, syn, stream=None):
        """(decision int32 [B], margin float64 [B]) on the device."""
        import torch
        self._check_det(syn)
        B = syn.shape[0]
        dec = torch.empty(B, dtype=torch.int32, device=syn.device)
        mar = torch.empty(B, dtype=torch.float64, device=syn.device)
        check(self._lib.td_gen_decode(self._h, C.c_void_p(syn.data_ptr()), B, C.c_void_p(dec.data_ptr()),
                                      C.c_void_p(mar.data_ptr()), self._stream(stream)))
        return dec, mar


def fma_peak_tflops(fp64: bool = True, iters: int = 1 << 16, stream=None) -> float:
    """td_measure_fma_peak: measured FMA throughput (TFLOP/s) of the current GPU."""
    import torch
    lib = load_library()
    out = C.c_double(0.0)
    s = stream if stream is not None else torch.cuda.current_stream()
    check(lib.td_measure_fma_peak(1 if fp64 else 0, int(iters), C.byref(out), C.c_void_p(s.cuda_stream)))
    return out.value


def mean_logprob(net: "Network", det, p):
    """(1/B) sum_b log P(m_b) as a differentiable function of the rates p (float64
    [n_mech] on det's device): the value and its gradient come from one td_grad_logprob
    call, so torch.autograd can drive a maximum-likelihood fit of the noise model."""
    import torch

    class _MeanLogProb(torch.autograd.Function):
        @staticmethod
        def forward(ctx, rates):
            logP, grad = net.grad_logprob(det, rates.detach())
            ctx.save_for_backward(grad)
            return logP.mean()

        @staticmethod
        def backward(ctx, g):
            (grad,) = ctx.saved_tensors
            return g * grad

    return _MeanLogProb.apply(p)

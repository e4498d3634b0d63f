"""Thin ctypes binding of ``libgwl.so`` (include/gwl.h): argument marshalling only.

Every computation runs in the library's CUDA kernels.  PyTorch supplies device
memory and streams.  If the compiled library is missing, importing this module
raises: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libgwl.so")

GWL_OK = 0
GWL_FP64 = 0
GWL_MIXED = 1
GWL_MIXED_F64PHASE = 2
GWL_FCUT_ISCO = 0
GWL_FCUT_BAND = 1
N_PARAM = 11
MAX_DET = 4

# exported symbols declared in include/gwl.h
EXPORTS = ("gwl_create", "gwl_loglike", "gwl_loglike_host", "gwl_loglike_static", "ns_run", "gwl_grad", "gwl_waveform", "ns_replace",
           "gwl_sync", "gwl_set_tuning", "gwl_profile", "gwl_profile_read", "gwl_device_bytes",
           "gwl_launch_count", "gwl_destroy", "gwl_last_error", "gwl_multi_create", "gwl_multi_loglike",
           "gwl_multi_ns_run", "gwl_multi_ns_run_resumable", "gwl_multi_ns_state_doubles",
           "gwl_multi_launch_count", "gwl_multi_destroy", "gwl_set_walk",
           "gwl_set_galilean", "ns_run_resumable", "ns_state_doubles", "gwl_get_tuning", "gwl_autotune", "gwl_set_calibration", "gwl_get_calibration", "gwl_ff_eval",
           "gwl_test_wait_timeout", "gwl_test_philox",
           "gwl_test_ffdelta_blocks")
GWL_WALK_RANDOM = 0
GWL_WALK_GALILEAN = 1
GWL_GALILEAN_PERSISTENCE = 0.5
KERNEL_PROLOGUE, KERNEL_BINS, KERNEL_COMBINE, KERNEL_GRAD, KERNEL_WALK, KERNEL_CALGRAD = range(6)
GWL_TUNE_LOGLIKE = 1
GWL_TUNE_GRAD = 2
GWL_BINS_AUTO, GWL_BINS_WARP, GWL_BINS_LANE = 1, 2, 3


class GwlDetector(C.Structure):
    _fields_ = [("vertex", C.c_double * 3), ("xarm", C.c_double * 3), ("yarm", C.c_double * 3)]


class GwlOptions(C.Structure):
    _fields_ = [
        ("precision", C.c_int),
        ("fcut_mode", C.c_int),
        ("gmst", C.c_double),
        ("t_ref", C.c_double),
        ("n_dim", C.c_int),
        ("param_map", C.c_int * N_PARAM),
        ("fixed_theta", C.c_double * N_PARAM),
        ("prior_kind", C.c_int * N_PARAM),
        ("prior_lo", C.c_double * N_PARAM),
        ("prior_hi", C.c_double * N_PARAM),
        ("periodic", C.c_int * N_PARAM),
    ]


class GwlNsResult(C.Structure):
    _fields_ = [("lnZ", C.c_double), ("lnZ_err", C.c_double), ("H", C.c_double), ("n_dead", C.c_int64),
                ("n_proposals", C.c_int64), ("rounds", C.c_int64), ("scale", C.c_double), ("acceptance", C.c_double),
                ("consumed_per_round", C.c_double), ("dlogz", C.c_double), ("n_dead_returned", C.c_int64)]


class GwlTuning(C.Structure):
    _fields_ = [("window", C.c_int), ("ctas_per_sm", C.c_int), ("grad_window", C.c_int),
                ("ms_loglike", C.c_double), ("ms_grad", C.c_double), ("n_tried", C.c_int), ("bin_kernel", C.c_int),
                ("lane_chunk", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class GwlError(RuntimeError):
    pass


_lib = None


def lib() -> C.CDLL:
    """Load the compiled library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise GwlError(f"{LIB_PATH} not found: build it with paper_1909_11873_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        P, i64, i32, d, u64 = C.c_void_p, C.c_int64, C.c_int, C.c_double, C.c_uint64
        L.gwl_create.argtypes = [P, i64, P, P, P, i32, C.POINTER(GwlOptions), C.POINTER(P)]
        L.gwl_loglike.argtypes = [P, P, i64, P, P]
        L.gwl_loglike_host.argtypes = [P, P, i64, P, P]
        L.gwl_loglike_static.argtypes = [P, P, i64, P, P]
        L.gwl_grad.argtypes = [P, P, i64, P, P, P]
        L.gwl_waveform.argtypes = [P, P, i64, P, P]
        L.ns_replace.argtypes = [P, P, P, i64, i64, d, u64, u64, i64, i32, d, P, P, P, P, P, P]
        L.ns_run.argtypes = [P, i64, i64, i32, u64, d, i64, d, i64, P, P, P, C.POINTER(GwlNsResult), P]
        L.ns_run_resumable.argtypes = [P, i64, i64, i32, u64, d, i64, d, i64, P, P, P, C.POINTER(GwlNsResult), P, P,
                                       P]
        L.ns_state_doubles.argtypes = [i64, i64, i64]
        L.ns_state_doubles.restype = i64
        L.gwl_sync.argtypes = [P]
        L.gwl_set_tuning.argtypes = [P, C.POINTER(GwlTuning)]
        L.gwl_get_tuning.argtypes = [P, C.POINTER(GwlTuning)]
        L.gwl_autotune.argtypes = [P, P, i64, i32, C.POINTER(GwlTuning), P]
        L.gwl_set_calibration.argtypes = [P, i32, P, d, d]
        L.gwl_ff_eval.argtypes = [P, i64, i32, P, P]
        L.gwl_test_wait_timeout.argtypes = [P, C.c_double, P]
        L.gwl_test_philox.argtypes = [P, i64, P, P]
        L.gwl_test_ffdelta_blocks.argtypes = [P, i32, C.POINTER(i64)]
        L.gwl_get_calibration.argtypes = [P, C.POINTER(i32), C.POINTER(i64)]
        L.gwl_set_walk.argtypes = [P, i32]
        L.gwl_set_galilean.argtypes = [P, C.c_double]
        L.gwl_profile.argtypes = [P, i32]
        L.gwl_profile_read.argtypes = [P, i32, C.POINTER(d), C.POINTER(i64)]
        L.gwl_device_bytes.argtypes = [P]
        L.gwl_device_bytes.restype = i64
        L.gwl_launch_count.argtypes = [P]
        L.gwl_launch_count.restype = i64
        L.gwl_destroy.argtypes = [P]
        L.gwl_destroy.restype = None
        L.gwl_last_error.restype = C.c_char_p
        L.gwl_multi_create.argtypes = [P, i32, C.POINTER(P)]
        L.gwl_multi_loglike.argtypes = [P, P, i64, P, P]
        L.gwl_multi_ns_run.argtypes = [P, i64, i64, i32, u64, d, i64, d, P, P]
        L.gwl_multi_ns_run_resumable.argtypes = [P, i64, i64, i32, u64, d, i64, d, P, P, P, P]
        L.gwl_multi_ns_state_doubles.argtypes = [P, i64]
        L.gwl_multi_ns_state_doubles.restype = i64
        L.gwl_multi_launch_count.argtypes = [P]
        L.gwl_multi_launch_count.restype = i64
        L.gwl_multi_destroy.argtypes = [P]
        L.gwl_multi_destroy.restype = None
        _lib = L
    return _lib


def _check(rc: int, what: str):
    if rc != GWL_OK:
        raise GwlError(f"{what} failed ({rc}): {lib().gwl_last_error().decode()}")


def _ptr(t) -> int:
    """Device or host address of a torch tensor / numpy array (contiguity checked)."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        if not t.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        if t.flags.writeable and t.nbytes:
            # the buffer's address without building numpy's ctypes helper object (about a
            # microsecond less per array on the host-buffer entry point)
            return C.addressof(C.c_char.from_buffer(t))
        return t.ctypes.data
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


def _stream(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return stream if isinstance(stream, int) else stream.cuda_stream


def detectors(geom: np.ndarray):
    g = np.asarray(geom, dtype=np.float64).reshape(-1, 9)
    arr = (GwlDetector * g.shape[0])()
    for i, row in enumerate(g):
        arr[i].vertex[:] = row[0:3].tolist()
        arr[i].xarm[:] = row[3:6].tolist()
        arr[i].yarm[:] = row[6:9].tolist()
    return arr


def options(precision: int, fcut_mode: int, gmst: float, t_ref: float, sampling) -> GwlOptions:
    o = GwlOptions()
    o.precision = precision
    o.fcut_mode = fcut_mode
    o.gmst = gmst
    o.t_ref = t_ref
    D = len(sampling.param_map)
    o.n_dim = D
    for i in range(D):
        o.param_map[i] = int(sampling.param_map[i])
        o.prior_kind[i] = int(sampling.kind[i])
        o.prior_lo[i] = float(sampling.lo[i])
        o.prior_hi[i] = float(sampling.hi[i])
        o.periodic[i] = int(sampling.periodic[i])
    for k in range(N_PARAM):
        o.fixed_theta[k] = float(sampling.fixed[k])
    return o


class Context:
    """One data segment on the current CUDA device (wraps a ``gwl_ctx*``)."""

    def __init__(self, freqs, strain, psd, geom, precision, fcut_mode, gmst, t_ref, sampling):
        fr = np.ascontiguousarray(freqs, dtype=np.float64)
        st = np.ascontiguousarray(np.stack([np.real(strain), np.imag(strain)], axis=-1), dtype=np.float64)
        ps = np.ascontiguousarray(psd, dtype=np.float64)
        dets = detectors(geom)
        self.opt = options(precision, fcut_mode, gmst, t_ref, sampling)
        self.n_dim = self.opt.n_dim
        self.n_det = len(dets)
        self.M = fr.size
        h = C.c_void_p()
        _check(lib().gwl_create(fr.ctypes.data, fr.size, st.ctypes.data, ps.ctypes.data, dets, len(dets),
                                C.byref(self.opt), C.byref(h)), "gwl_create")
        self._h = h

    @classmethod
    def from_event(cls, ev, precision=GWL_MIXED, sampling=None):
        return cls(ev.freqs, ev.strain, ev.psd, ev.geom, precision, ev.fcut_mode, ev.gmst, ev.t_ref,
                   sampling if sampling is not None else ev.sampling)

    @property
    def handle(self) -> int:
        return self._h.value

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().gwl_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- compute entry points (same names as the C ABI)
    def gwl_loglike(self, theta, lnl, stream=None):
        _check(lib().gwl_loglike(self._h, _ptr(theta), theta.shape[0], _ptr(lnl), _stream(stream)), "gwl_loglike")

    def gwl_loglike_host(self, theta: np.ndarray, lnl: np.ndarray, stream=None):
        _check(lib().gwl_loglike_host(self._h, _ptr(theta), theta.shape[0], _ptr(lnl), _stream(stream)),
               "gwl_loglike_host")

    def gwl_loglike_static(self, theta, lnl, stream=None):
        """gwl_loglike with its scratch in the library's fixed device array (no allocation)."""
        _check(lib().gwl_loglike_static(self._h, _ptr(theta), theta.shape[0], _ptr(lnl), _stream(stream)),
               "gwl_loglike_static")

    def gwl_grad(self, theta, lnl, grad, stream=None):
        _check(lib().gwl_grad(self._h, _ptr(theta), theta.shape[0], _ptr(lnl), _ptr(grad), _stream(stream)),
               "gwl_grad")

    def gwl_waveform(self, theta, h, stream=None):
        _check(lib().gwl_waveform(self._h, _ptr(theta), theta.shape[0], _ptr(h), _stream(stream)), "gwl_waveform")

    def ns_replace(self, live_u, live_lnl, worst, lnl_star, seed, counter, n_chains, walk_len, scale, chol,
                   out_u, out_lnl, out_nacc, out_start=None, stream=None):
        _check(lib().ns_replace(self._h, _ptr(live_u), _ptr(live_lnl), live_u.shape[0], int(worst), float(lnl_star),
                                int(seed), int(counter), int(n_chains), int(walk_len), float(scale), _ptr(chol),
                                _ptr(out_u), _ptr(out_lnl), _ptr(out_nacc), _ptr(out_start), _stream(stream)),
               "ns_replace")

    def ns_run(self, K, n_chains, walk_len, seed, dlogz=0.1, max_rounds=100000, scale0=1.0, max_dead=0,
               stream=None, resume=None, checkpoint=False):
        """Static parallel nested sampling on the device; returns a dict (plus dead points if max_dead > 0).
        resume: a checkpoint (float64 array) to continue from; checkpoint=True adds the state after this call's
        rounds as out["state"] (ns_run_resumable)."""
        r = GwlNsResult()
        D = self.theta_stride
        dl = np.zeros(max(max_dead, 1))
        dw = np.zeros(max(max_dead, 1))
        du = np.zeros((max(max_dead, 1), D))
        res = None if resume is None else np.ascontiguousarray(resume, dtype=np.float64)
        state = np.zeros(lib().ns_state_doubles(int(K), D, int(max_dead))) if checkpoint else None
        _check(lib().ns_run_resumable(self._h, int(K), int(n_chains), int(walk_len), int(seed), float(dlogz),
                                      int(max_rounds), float(scale0), int(max_dead),
                                      dl.ctypes.data if max_dead else None, dw.ctypes.data if max_dead else None,
                                      du.ctypes.data if max_dead else None, C.byref(r),
                                      None if res is None else res.ctypes.data,
                                      None if state is None else state.ctypes.data, _stream(stream)),
               "ns_run_resumable")
        out = {k: getattr(r, k) for k, _ in GwlNsResult._fields_}
        if max_dead:
            n = r.n_dead_returned
            out.update(dead_lnl=dl[:n], dead_logwt=dw[:n], dead_u=du[:n])
        if checkpoint:
            out["state"] = state
        return out

    def ns_run_checkpointed(self, path, K, n_chains, walk_len, seed, every, dlogz=0.1, max_rounds=100000,
                            scale0=1.0, max_dead=0):
        """ns_run in calls of `every` rounds, the state written to the .npz file `path` after each; a run whose
        file exists continues from it.  Returns the last call's result (the whole run's)."""
        import os
        state, before = None, 0
        if os.path.exists(path):
            f = np.load(path)
            state, before = f["state"], int(f["rounds"])
        while True:
            todo = max(min(every, max_rounds - before), 0)
            out = self.ns_run(K, n_chains, walk_len, seed, dlogz, todo, scale0, max_dead, resume=state,
                              checkpoint=True)
            state = out.pop("state")
            tmp = path + ".tmp.npz"
            np.savez(tmp, state=state, rounds=out["rounds"])
            os.replace(tmp, path)
            if out["rounds"] - before < todo or out["rounds"] >= max_rounds or todo == 0:
                return out
            before = out["rounds"]

    def gwl_sync(self):
        _check(lib().gwl_sync(self._h), "gwl_sync")

    def gwl_test_wait_timeout(self, seconds: float, stream=None):
        _check(lib().gwl_test_wait_timeout(self._h, float(seconds), _stream(stream)), "gwl_test_wait_timeout")

    def gwl_test_ffdelta_blocks(self, enable: int = -1) -> int:
        """Blocks counted so far that took the float-float phase delta; then enable (1), stop (0) or keep (-1)."""
        n = C.c_int64()
        _check(lib().gwl_test_ffdelta_blocks(self._h, int(enable), C.byref(n)), "gwl_test_ffdelta_blocks")
        return int(n.value)

    def gwl_set_walk(self, kind: int):
        _check(lib().gwl_set_walk(self._h, int(kind)), "gwl_set_walk")

    def gwl_set_galilean(self, persistence: float):
        _check(lib().gwl_set_galilean(self._h, float(persistence)), "gwl_set_galilean")

    def gwl_set_tuning(self, window=0, ctas_per_sm=0, grad_window=0, bin_kernel=0, lane_chunk=0):
        t = GwlTuning(int(window), int(ctas_per_sm), int(grad_window), 0.0, 0.0, 0, int(bin_kernel), int(lane_chunk))
        _check(lib().gwl_set_tuning(self._h, C.byref(t)), "gwl_set_tuning")

    def gwl_get_tuning(self) -> dict:
        t = GwlTuning()
        _check(lib().gwl_get_tuning(self._h, C.byref(t)), "gwl_get_tuning")
        return t.as_dict()

    def gwl_autotune(self, theta, what=GWL_TUNE_LOGLIKE | GWL_TUNE_GRAD, stream=None) -> dict:
        """Time the bin-loop launch shapes on this batch (B x n_dim, float64, on the device); keep the fastest."""
        t = GwlTuning()
        _check(lib().gwl_autotune(self._h, _ptr(theta), theta.shape[0], int(what), C.byref(t), _stream(stream)),
               "gwl_autotune")
        return t.as_dict()

    def gwl_set_calibration(self, node_freqs, sigma_amp=0.1, sigma_phase=0.1):
        """Calibration model at these node frequencies [Hz] (empty: off); rows of theta then hold
        n_dim + 2 n_nodes n_det values (per detector dA at the nodes, then dphi), and ns_replace /
        ns_run sample them under zero-mean Gaussian priors of these widths."""
        nf = np.ascontiguousarray(node_freqs, dtype=np.float64).ravel()
        _check(lib().gwl_set_calibration(self._h, nf.size, nf.ctypes.data if nf.size else None, float(sigma_amp),
                                         float(sigma_phase)), "gwl_set_calibration")

    def gwl_get_calibration(self):
        """(calibration nodes, doubles per row of theta)."""
        n = C.c_int()
        st = C.c_int64()
        _check(lib().gwl_get_calibration(self._h, C.byref(n), C.byref(st)), "gwl_get_calibration")
        return n.value, st.value

    @property
    def theta_stride(self) -> int:
        return self.gwl_get_calibration()[1]

    def gwl_profile(self, enable: bool):
        _check(lib().gwl_profile(self._h, int(bool(enable))), "gwl_profile")

    def gwl_profile_read(self, kind: int):
        """(total device ms, launch count) of one kernel class since profiling was enabled."""
        ms = C.c_double()
        n = C.c_int64()
        _check(lib().gwl_profile_read(self._h, int(kind), C.byref(ms), C.byref(n)), "gwl_profile_read")
        return ms.value, n.value

    def device_bytes(self) -> int:
        return lib().gwl_device_bytes(self._h)

    def launch_count(self) -> int:
        return lib().gwl_launch_count(self._h)


GWL_FF_EXP, GWL_FF_LOG, GWL_FF_SIN, GWL_FF_COS, GWL_F32_SINPI, GWL_F32_COSPI = range(6)


def ff_eval(x, fn, stream=None):
    """The library's float-float exp / log / sin / cos (GWL_FF_*), or the FP32 sin(pi x) / cos(pi x) of the
    gradient's bin loop (GWL_F32_*), of a float64 CUDA tensor."""
    import torch
    out = torch.empty_like(x)
    _check(lib().gwl_ff_eval(_ptr(x), x.numel(), int(fn), _ptr(out), _stream(stream)), "gwl_ff_eval")
    return out


def philox_eval(records, stream=None):
    """The device Philox4x32-10 on an int64 CUDA tensor [n][6] of 32-bit words (counter c0..c3, key k0, k1);
    returns the [n][4] output words (int64)."""
    import torch
    inp = records.to(torch.int32).contiguous()
    out = torch.empty((inp.shape[0], 4), dtype=torch.int32, device=inp.device)
    _check(lib().gwl_test_philox(_ptr(inp), inp.shape[0], _ptr(out), _stream(stream)), "gwl_test_philox")
    return out.to(torch.int64) & 0xFFFFFFFF


# ---- convenience wrappers used by tests and the benchmark (torch tensors in, torch tensors out)
def loglike(ctx: Context, theta, stream=None):
    import torch
    out = torch.empty(theta.shape[0], dtype=torch.float64, device=theta.device)
    ctx.gwl_loglike(theta, out, stream)
    return out


def waveform(ctx: Context, theta, stream=None):
    import torch
    out = torch.empty((theta.shape[0], ctx.n_det, ctx.M, 2), dtype=torch.float64, device=theta.device)
    ctx.gwl_waveform(theta, out, stream)
    return out


def grad(ctx: Context, theta, stream=None):
    """(lnL [B], d lnL / d theta [B, theta_stride]) via gwl_grad (theta_stride: n_dim, plus the
    calibration parameters with the calibration model)."""
    import torch
    out = torch.empty(theta.shape[0], dtype=torch.float64, device=theta.device)
    g = torch.empty_like(theta)
    ctx.gwl_grad(theta, out, g, stream)
    return out, g


_GWLogLike = None


def GWLogLike():
    """torch.autograd.Function: lnL(theta) with the gradient from the adjoint kernel.

    Usage: ``lnl = GWLogLike().apply(theta, ctx)``; forward runs gwl_grad when
    theta requires a gradient (gwl_loglike otherwise) and backward scales the
    stored gradient rows by the incoming gradient.
    """
    global _GWLogLike
    if _GWLogLike is None:
        import torch

        class _F(torch.autograd.Function):
            @staticmethod
            def forward(fctx, theta, gctx):
                th = theta.detach().contiguous()
                if theta.requires_grad:
                    lnl, g = grad(gctx, th)
                    fctx.save_for_backward(g)
                else:
                    lnl = loglike(gctx, th)
                return lnl

            @staticmethod
            def backward(fctx, gout):
                (g,) = fctx.saved_tensors
                return gout[:, None] * g, None

        _GWLogLike = _F
    return _GWLogLike


class MultiContext:
    """Several events evaluated in one batch (wraps a ``gwl_multi*``); keeps its contexts alive."""

    def __init__(self, contexts):
        self.contexts = list(contexts)
        arr = (C.c_void_p * len(self.contexts))(*[c.handle for c in self.contexts])
        h = C.c_void_p()
        _check(lib().gwl_multi_create(arr, len(self.contexts), C.byref(h)), "gwl_multi_create")
        self._h = h
        self.E = len(self.contexts)
        self.n_dim = self.contexts[0].n_dim

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().gwl_multi_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def gwl_multi_loglike(self, theta, lnl, stream=None):
        """theta [E * n_per, theta_stride] (event-major; theta_stride = n_dim plus the calibration parameters),
        lnl [E * n_per]."""
        n_per = theta.shape[0] // self.E
        _check(lib().gwl_multi_loglike(self._h, _ptr(theta), n_per, _ptr(lnl), _stream(stream)), "gwl_multi_loglike")

    def gwl_multi_ns_run(self, K, n_chains, walk_len, seed, dlogz=0.1, max_rounds=100000, scale0=1.0, stream=None,
                         resume=None, checkpoint=False):
        """ns_run for every event in one graph per round; a list of per-event results.  resume: a checkpoint
        (float64 array) to continue from; checkpoint=True returns (results, state) with the state after this
        call's rounds (gwl_multi_ns_run_resumable)."""
        res = (GwlNsResult * self.E)()
        state = np.zeros(lib().gwl_multi_ns_state_doubles(self._h, int(K))) if checkpoint else None
        if resume is not None:
            resume = np.ascontiguousarray(resume, dtype=np.float64)
        _check(lib().gwl_multi_ns_run_resumable(self._h, int(K), int(n_chains), int(walk_len), int(seed),
                                                float(dlogz), int(max_rounds), float(scale0),
                                                C.cast(res, C.c_void_p), _ptr(resume), _ptr(state),
                                                _stream(stream)),
               "gwl_multi_ns_run_resumable")
        out = [{k: getattr(r, k) for k, _ in GwlNsResult._fields_} for r in res]
        return (out, state) if checkpoint else out

    def launch_count(self) -> int:
        return lib().gwl_multi_launch_count(self._h)

"""Python binding of the FEWHA C ABI (include/fewha.h).

Argument marshalling only: every operator runs in the CUDA library
``libfewha.so`` built in-tree for sm_103a.  PyTorch supplies device memory and
streams.  There is no CPU fallback: if the library or a CUDA device is missing,
the constructor raises.
"""

import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libfewha.so")

FLAG_GRAPH = 1
FLAG_WARM_RESIDUAL = 2
FLAG_PDL = 4
FLAG_AUGMENTED = 8
FLAG_CLOSED_LOOP = 16
FLAG_PERSISTENT = 32
AUG_MAX_ITERS = 8

ERRORS = {
    -1: "invalid argument",
    -2: "geometry",
    -3: "out of device memory",
    -4: "CUDA error",
    -5: "non-finite input",
    -6: "size limit",
    -7: "a grid-wide wait ran out",
}


class FewhaError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("FEWHA error %d (%s): %s" % (code, ERRORS.get(code, "?"), msg))
        self.code = code


class Telescope(ctypes.Structure):
    _fields_ = [("D", ctypes.c_double), ("obs", ctypes.c_double)]


class Wfs(ctypes.Structure):
    _fields_ = [("n_sub", ctypes.c_int), ("nb", ctypes.c_int), ("is_lgs", ctypes.c_int),
                ("theta_x", ctypes.c_double), ("theta_y", ctypes.c_double),
                ("H", ctypes.c_double), ("sigma", ctypes.c_double),
                ("launch_x", ctypes.c_double), ("launch_y", ctypes.c_double),
                ("na_fwhm", ctypes.c_double), ("spot_fwhm", ctypes.c_double)]


class Layer(ctypes.Structure):
    _fields_ = [("h", ctypes.c_double), ("cn2_weight", ctypes.c_double),
                ("spacing", ctypes.c_double), ("n", ctypes.c_int), ("levels", ctypes.c_int)]


class Dm(ctypes.Structure):
    _fields_ = [("h", ctypes.c_double), ("spacing", ctypes.c_double), ("n_act", ctypes.c_int)]


class Params(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("tau", ctypes.c_double), ("gain", ctypes.c_double),
                ("r0", ctypes.c_double), ("L0", ctypes.c_double), ("iters", ctypes.c_int),
                ("precision", ctypes.c_int), ("flags", ctypes.c_uint),
                ("alpha_eta", ctypes.c_double), ("warm_refresh", ctypes.c_int)]


class LsFit(ctypes.Structure):
    _fields_ = [("n_dirs", ctypes.c_int), ("theta_x", ctypes.POINTER(ctypes.c_double)),
                ("theta_y", ctypes.POINTER(ctypes.c_double)), ("weight", ctypes.POINTER(ctypes.c_double)),
                ("n_fit", ctypes.c_int), ("eps", ctypes.c_double)]


class BatchConfig(ctypes.Structure):
    _fields_ = [("order", ctypes.c_int), ("groups", ctypes.c_int), ("vec_passes", ctypes.c_int),
                ("pair_threads", ctypes.c_int), ("proj_taps", ctypes.c_int), ("vec_threads", ctypes.c_int)]


_VP = ctypes.c_void_p
_OPS = ["fewha_apply_M", "fewha_rhs", "fewha_dwt", "fewha_idwt", "fewha_project",
        "fewha_project_adj", "fewha_slopes", "fewha_slopes_adj", "fewha_noise_weight",
        "fewha_forward", "fewha_forward_adj", "fewha_fit", "fewha_fit_adj"]
EXPORTS = ["fewha_create", "fewha_destroy", "fewha_last_error", "fewha_create_error",
           "fewha_sizes", "fewha_update_params", "fewha_reset", "fewha_reconstruct",
           "fewha_reconstruct_f64", "fewha_reconstruct_host", "fewha_reconstruct_host_f64",
           "fewha_check_input", "fewha_pcg", "fewha_get_diagonals", "fewha_bench_stage",
           "fewha_frame_launches", "fewha_apply_M_noalloc", "fewha_run_loop",
           "fewha_run_loop_f64", "fewha_batch_create", "fewha_batch_destroy",
           "fewha_batch_last_error", "fewha_batch_set_config", "fewha_batch_get_config",
           "fewha_batch_reconstruct", "fewha_batch_autotune", "fewha_reconstruct_batched",
           "fewha_reconstruct_batched_f64", "fewha_get_state", "fewha_set_state", "fewha_solve",
           "fewha_reconstruct_converged", "fewha_backward", "fewha_get_residual", "fewha_frame_vjp",
           "fewha_set_wait_limit", "fewha_device_bytes", "fewha_test_fail_alloc", "fewha_fit_ls"] + _OPS

STAGES = {"idwt": 0, "sensor": 1, "layer": 2, "vector": 3, "rhs": 4, "fit": 5, "proj": 6,
          "projT": 7}

_lib = None


def lib():
    """Load libfewha.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libfewha.so is missing: run `python -m paper_2202_11945_gb300.build`")
    L = ctypes.CDLL(LIB_PATH)
    L.fewha_create.argtypes = [ctypes.POINTER(Telescope), ctypes.POINTER(Wfs), ctypes.c_int,
                               ctypes.POINTER(Layer), ctypes.c_int, ctypes.POINTER(Dm),
                               ctypes.c_int, ctypes.POINTER(Params), ctypes.POINTER(_VP)]
    L.fewha_create.restype = ctypes.c_int
    L.fewha_destroy.argtypes = [_VP]
    L.fewha_destroy.restype = None
    L.fewha_last_error.argtypes = [_VP]
    L.fewha_last_error.restype = ctypes.c_char_p
    L.fewha_create_error.argtypes = []
    L.fewha_create_error.restype = ctypes.c_char_p
    i64p = ctypes.POINTER(ctypes.c_int64)
    L.fewha_sizes.argtypes = [_VP, i64p, i64p, i64p, i64p]
    L.fewha_update_params.argtypes = [_VP, ctypes.POINTER(Params), _VP, _VP]
    L.fewha_reset.argtypes = [_VP, _VP]
    for name in ["fewha_reconstruct", "fewha_reconstruct_f64"]:
        getattr(L, name).argtypes = [_VP, _VP, _VP, _VP, _VP]
    for name in ["fewha_reconstruct_host", "fewha_reconstruct_host_f64"]:
        getattr(L, name).argtypes = [_VP, _VP, _VP, _VP]
    L.fewha_check_input.argtypes = [_VP, ctypes.POINTER(ctypes.c_int), _VP]
    L.fewha_pcg.argtypes = [_VP, _VP, _VP, ctypes.c_int, _VP]
    L.fewha_get_diagonals.argtypes = [_VP, _VP, _VP, _VP]
    L.fewha_bench_stage.argtypes = [_VP, ctypes.c_int, ctypes.c_int, _VP]
    L.fewha_frame_launches.argtypes = [_VP, ctypes.POINTER(ctypes.c_int)]
    L.fewha_set_wait_limit.argtypes = [_VP, ctypes.c_uint, ctypes.c_uint]
    L.fewha_device_bytes.argtypes = [_VP, ctypes.POINTER(ctypes.c_int64)]
    L.fewha_test_fail_alloc.argtypes = [ctypes.c_int]
    ip, dp = ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)
    for name in ["fewha_solve", "fewha_reconstruct_converged"]:
        getattr(L, name).argtypes = [_VP, _VP, _VP, ctypes.c_double, ctypes.c_int, ip, dp, _VP]
    L.fewha_backward.argtypes = [_VP, _VP, _VP, dp, dp, _VP]
    L.fewha_fit_ls.argtypes = [_VP, ctypes.POINTER(LsFit), _VP, _VP, ctypes.c_double, ctypes.c_int, ip, dp, _VP]
    L.fewha_get_state.argtypes = [_VP, _VP, _VP, _VP]
    L.fewha_set_state.argtypes = [_VP, _VP, _VP, _VP]
    L.fewha_get_residual.argtypes = [_VP, _VP, _VP, _VP]
    L.fewha_frame_vjp.argtypes = [_VP, _VP, _VP, _VP, _VP, _VP, _VP]
    for name in ["fewha_run_loop", "fewha_run_loop_f64"]:
        getattr(L, name).argtypes = [_VP, _VP, ctypes.c_int, _VP, ctypes.c_double, _VP, _VP,
                                     ctypes.POINTER(ctypes.c_int), _VP]
    for name in _OPS + ["fewha_apply_M_noalloc"]:
        getattr(L, name).argtypes = [_VP, _VP, _VP, _VP]
    L.fewha_batch_create.argtypes = [ctypes.POINTER(_VP), ctypes.c_int, ctypes.POINTER(_VP)]
    L.fewha_batch_destroy.argtypes = [_VP]
    L.fewha_batch_destroy.restype = None
    L.fewha_batch_last_error.argtypes = [_VP]
    L.fewha_batch_last_error.restype = ctypes.c_char_p
    L.fewha_batch_set_config.argtypes = [_VP, ctypes.POINTER(BatchConfig)]
    L.fewha_batch_get_config.argtypes = [_VP, ctypes.POINTER(BatchConfig)]
    L.fewha_batch_reconstruct.argtypes = [_VP, ctypes.POINTER(_VP), ctypes.POINTER(_VP), _VP]
    L.fewha_batch_autotune.argtypes = [_VP, ctypes.POINTER(_VP), ctypes.POINTER(_VP), ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_float), _VP]
    for name in ["fewha_reconstruct_batched", "fewha_reconstruct_batched_f64"]:
        getattr(L, name).argtypes = [ctypes.POINTER(_VP), ctypes.c_int, ctypes.POINTER(_VP),
                                     ctypes.POINTER(_VP), _VP]
    for name in EXPORTS:
        if name not in ("fewha_destroy", "fewha_last_error", "fewha_create_error",
                        "fewha_batch_destroy", "fewha_batch_last_error"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def structs_from_workload(wl, precision=32, flags=FLAG_GRAPH):
    """C structs of a workload description (see synth.configs for the dict format)."""
    tel = Telescope(wl["D"], wl["obs"])
    wfs = (Wfs * len(wl["wfs"]))(*[
        Wfs(w["n_sub"], w["nb"], 1 if w["lgs"] else 0, w["theta"][0], w["theta"][1],
            w["H"] if w["lgs"] else 0.0, w["sigma"], *w.get("launch", (0.0, 0.0)),
            w.get("na_fwhm", 0.0), w.get("spot_fwhm", 0.0)) for w in wl["wfs"]])
    layers = (Layer * len(wl["layers"]))(*[
        Layer(L["h"], L["w"], L["delta"], L["n"], L["levels"]) for L in wl["layers"]])
    dms = (Dm * len(wl["dms"]))(*[Dm(m["h"], m["spacing"], m["n_act"]) for m in wl["dms"]])
    p = wl["params"]
    params = Params(p["alpha"], p.get("tau", 0.0), p.get("gain", 1.0), p["r0"], p["L0"],
                    p["iters"], precision, flags, p.get("alpha_eta", 0.0), p.get("warm_refresh", 0))
    return tel, wfs, layers, dms, params


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Reconstructor:
    """One FEWHA instance on the current CUDA device (a handle of the C library)."""

    def __init__(self, wl, precision=32, graph=True, warm_residual=False, pdl=True, augmented=False,
                 closed_loop=False, persistent=False, warm_refresh=0):
        if not torch.cuda.is_available():
            raise RuntimeError("FEWHA needs a CUDA device; there is no CPU path")
        torch.cuda.init()
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.precision = precision
        self.dtype = torch.float32 if precision == 32 else torch.float64
        flags = ((FLAG_GRAPH if graph else 0) | (FLAG_WARM_RESIDUAL if warm_residual else 0) |
                 (FLAG_PDL if pdl else 0) | (FLAG_AUGMENTED if augmented else 0) |
                 (FLAG_CLOSED_LOOP if closed_loop else 0) | (FLAG_PERSISTENT if persistent else 0))
        self._structs = structs_from_workload(wl, precision, flags)
        self._structs[4].warm_refresh = int(warm_refresh)
        tel, wfs, layers, dms, params = self._structs
        self.L = lib()
        h = _VP()
        rc = self.L.fewha_create(ctypes.byref(tel), wfs, len(wfs), layers, len(layers), dms,
                                 len(dms), ctypes.byref(params), ctypes.byref(h))
        if rc != 0:
            raise FewhaError(rc, self.L.fewha_create_error().decode())
        self.h = h
        ns, nc, na, nn = (ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64())
        self._check(self.L.fewha_sizes(h, ctypes.byref(ns), ctypes.byref(nc), ctypes.byref(na),
                                       ctypes.byref(nn)))
        self.n_slopes, self.n_coeffs, self.n_act, self.n_nodes = ns.value, nc.value, na.value, nn.value

    @property
    def iters(self):
        """PCG iterations per frame."""
        return self._structs[4].iters

    # -- plumbing ---------------------------------------------------------------
    def _check(self, rc):
        if rc != 0:
            raise FewhaError(rc, self.L.fewha_last_error(self.h).decode())

    def _dev(self, t, n, name):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == self.dtype
                and t.is_contiguous() and t.numel() == n):
            raise ValueError("%s must be a contiguous %s CUDA tensor of %d elements"
                             % (name, self.dtype, n))
        return ctypes.c_void_p(t.data_ptr())

    def _new(self, n):
        return torch.empty(n, dtype=self.dtype, device=self.device)

    def close(self):
        if getattr(self, "h", None):
            self.L.fewha_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- frame ------------------------------------------------------------------
    def reconstruct(self, slopes, x_warm=None, dm_out=None, stream=None):
        """One frame of Algorithm 1 on device tensors; returns the DM commands."""
        if dm_out is None:
            dm_out = self._new(self.n_act)
        s = self._dev(slopes, self.n_slopes, "slopes")
        x = self._dev(x_warm, self.n_coeffs, "x_warm") if x_warm is not None else None
        d = self._dev(dm_out, self.n_act, "dm_out")
        fn = self.L.fewha_reconstruct if self.precision == 32 else self.L.fewha_reconstruct_f64
        self._check(fn(self.h, s, x, d, _stream(stream)))
        return dm_out

    def reconstruct_host(self, slopes, dm_out, stream=None):
        """One frame from and to host tensors (copies inside the call; synchronous)."""
        for t, n, name in ((slopes, self.n_slopes, "slopes"), (dm_out, self.n_act, "dm_out")):
            if t.is_cuda or t.dtype != self.dtype or not t.is_contiguous() or t.numel() != n:
                raise ValueError("%s must be a contiguous host %s tensor of %d" % (name, self.dtype, n))
        fn = self.L.fewha_reconstruct_host if self.precision == 32 else self.L.fewha_reconstruct_host_f64
        self._check(fn(self.h, ctypes.c_void_p(slopes.data_ptr()), ctypes.c_void_p(dm_out.data_ptr()),
                       _stream(stream)))
        return dm_out

    def run_loop(self, slopes, period_us=1000.0, stream=None):
        """Frames of a real-time loop from host slopes (n_frames x n_slopes, any layout that
        converts to a contiguous host tensor of the handle's dtype), released every
        `period_us` (0: back to back), each warm-started from the previous one.

        Returns (dm [n_frames, n_act] host tensor, wall_us, device_us, n_late): per-frame
        host-clock latency from release to commands on the host, the CUDA-event time of
        the frame's copies and kernels, and the number of frames that missed the next
        release."""
        s = torch.as_tensor(slopes, dtype=self.dtype).contiguous()
        if s.is_cuda or s.dim() != 2 or s.shape[1] != self.n_slopes:
            raise ValueError("slopes must be a host array of shape [n_frames, %d]" % self.n_slopes)
        F = s.shape[0]
        s = s.pin_memory()
        dm = torch.empty((F, self.n_act), dtype=self.dtype).pin_memory()
        wall = torch.zeros(F, dtype=torch.float32)
        dev = torch.zeros(F, dtype=torch.float32)
        late = ctypes.c_int(0)
        fn = self.L.fewha_run_loop if self.precision == 32 else self.L.fewha_run_loop_f64
        self._check(fn(self.h, ctypes.c_void_p(s.data_ptr()), int(F), ctypes.c_void_p(dm.data_ptr()),
                       float(period_us), ctypes.c_void_p(wall.data_ptr()),
                       ctypes.c_void_p(dev.data_ptr()), ctypes.byref(late), _stream(stream)))
        return dm, wall, dev, late.value

    def get_state(self, stream=None):
        """(c, a_prev): copies of the warm-start coefficients and previous commands."""
        c, a = self._new(self.n_coeffs), self._new(self.n_act)
        self._check(self.L.fewha_get_state(self.h, self._dev(c, self.n_coeffs, "c"),
                                           self._dev(a, self.n_act, "a_prev"), _stream(stream)))
        return c, a

    def set_state(self, c=None, a_prev=None, stream=None):
        """Restore a saved state (either part may be None); the next frame forms its
        initial residual explicitly."""
        cp = self._dev(c, self.n_coeffs, "c") if c is not None else None
        ap = self._dev(a_prev, self.n_act, "a_prev") if a_prev is not None else None
        self._check(self.L.fewha_set_state(self.h, cp, ap, _stream(stream)))

    def residual(self, with_b=True, stream=None):
        """(r, b): the last frame's PCG residual and right-hand side (copies).  b exists only
        for the warm-residual, augmented and persistent frames (the plain explicit frame
        never forms it: use rhs(slopes)); with_b=False returns (r, None)."""
        r = self._new(self.n_coeffs)
        b = self._new(self.n_coeffs) if with_b else None
        self._check(self.L.fewha_get_residual(self.h, self._dev(r, self.n_coeffs, "r"),
                                              self._dev(b, self.n_coeffs, "b") if with_b else None,
                                              _stream(stream)))
        return r, b

    def frame_vjp(self, slopes, c0, grad_dm=None, stream=None):
        """The fixed-iteration frame from the warm start c0 (explicit initial residual, no
        control law) and, with grad_dm = dJ/da~, dJ/dslopes by reverse mode through the
        recurrence.  Returns (a~, dJ/dslopes or None)."""
        a = self._new(self.n_act)
        g = self._new(self.n_slopes) if grad_dm is not None else None
        gp = self._dev(grad_dm, self.n_act, "grad_dm") if grad_dm is not None else None
        self._check(self.L.fewha_frame_vjp(self.h, self._dev(slopes, self.n_slopes, "slopes"),
                                           self._dev(c0, self.n_coeffs, "c0"), gp,
                                           self._dev(a, self.n_act, "dm"),
                                           self._dev(g, self.n_slopes, "grad") if g is not None else None,
                                           _stream(stream)))
        return a, g

    def check_input(self, stream=None):
        flag = ctypes.c_int(0)
        self._check(self.L.fewha_check_input(self.h, ctypes.byref(flag), _stream(stream)))
        return bool(flag.value)

    def reset(self, stream=None):
        self._check(self.L.fewha_reset(self.h, _stream(stream)))

    def update_params(self, alpha=None, tau=None, gain=None, r0=None, L0=None, iters=None, alpha_eta=None,
                      cn2_weights=None, sigmas=None, graph=None, warm_residual=None, augmented=None,
                      closed_loop=None, warm_refresh=None):
        tel, wfs, layers, dms, p = self._structs
        if alpha is not None:
            p.alpha = alpha
        if tau is not None:
            p.tau = tau
        if gain is not None:
            p.gain = gain
        if r0 is not None:
            p.r0 = r0
        if L0 is not None:
            p.L0 = L0
        if iters is not None:
            p.iters = iters
        if alpha_eta is not None:
            p.alpha_eta = alpha_eta
        if warm_refresh is not None:
            p.warm_refresh = int(warm_refresh)
        if graph is not None:
            p.flags = (p.flags & ~FLAG_GRAPH) | (FLAG_GRAPH if graph else 0)
        if warm_residual is not None:
            p.flags = (p.flags & ~FLAG_WARM_RESIDUAL) | (FLAG_WARM_RESIDUAL if warm_residual else 0)
        if augmented is not None:
            p.flags = (p.flags & ~FLAG_AUGMENTED) | (FLAG_AUGMENTED if augmented else 0)
        if closed_loop is not None:
            p.flags = (p.flags & ~FLAG_CLOSED_LOOP) | (FLAG_CLOSED_LOOP if closed_loop else 0)
        w = s = None
        if cn2_weights is not None:
            w = (ctypes.c_double * len(layers))(*cn2_weights)
        if sigmas is not None:
            s = (ctypes.c_double * len(wfs))(*sigmas)
        self._check(self.L.fewha_update_params(self.h, ctypes.byref(p), w, s))

    # -- operators ----------------------------------------------------------------
    def _op(self, name, x, n_in, n_out, out=None, stream=None):
        if out is None:
            out = self._new(n_out)
        self._check(getattr(self.L, name)(self.h, self._dev(x, n_in, "input"),
                                          self._dev(out, n_out, "output"), _stream(stream)))
        return out

    def apply_M(self, c, out=None, stream=None):
        return self._op("fewha_apply_M", c, self.n_coeffs, self.n_coeffs, out, stream)

    def apply_M_noalloc(self, c, out=None, stream=None):
        """q = M c with the library's static scratch block (see fewha_apply_M_noalloc)."""
        return self._op("fewha_apply_M_noalloc", c, self.n_coeffs, self.n_coeffs, out, stream)

    def rhs(self, s, out=None, stream=None):
        return self._op("fewha_rhs", s, self.n_slopes, self.n_coeffs, out, stream)

    def dwt(self, phi, out=None, stream=None):
        return self._op("fewha_dwt", phi, self.n_coeffs, self.n_coeffs, out, stream)

    def idwt(self, c, out=None, stream=None):
        return self._op("fewha_idwt", c, self.n_coeffs, self.n_coeffs, out, stream)

    def project(self, phi, out=None, stream=None):
        return self._op("fewha_project", phi, self.n_coeffs, self.n_nodes, out, stream)

    def project_adj(self, v, out=None, stream=None):
        return self._op("fewha_project_adj", v, self.n_nodes, self.n_coeffs, out, stream)

    def slopes(self, v, out=None, stream=None):
        return self._op("fewha_slopes", v, self.n_nodes, self.n_slopes, out, stream)

    def slopes_adj(self, s, out=None, stream=None):
        return self._op("fewha_slopes_adj", s, self.n_slopes, self.n_nodes, out, stream)

    def noise_weight(self, s, out=None, stream=None):
        return self._op("fewha_noise_weight", s, self.n_slopes, self.n_slopes, out, stream)

    def forward(self, phi, out=None, stream=None):
        return self._op("fewha_forward", phi, self.n_coeffs, self.n_slopes, out, stream)

    def forward_adj(self, s, out=None, stream=None):
        return self._op("fewha_forward_adj", s, self.n_slopes, self.n_coeffs, out, stream)

    def fit(self, c, out=None, stream=None):
        return self._op("fewha_fit", c, self.n_coeffs, self.n_act, out, stream)

    def fit_adj(self, a, out=None, stream=None):
        return self._op("fewha_fit_adj", a, self.n_act, self.n_coeffs, out, stream)

    def pcg(self, b, c, iters, stream=None):
        """`iters` PCG iterations on M c = b, c updated in place."""
        self._check(self.L.fewha_pcg(self.h, self._dev(b, self.n_coeffs, "b"),
                                     self._dev(c, self.n_coeffs, "c"), int(iters), _stream(stream)))
        return c

    # -- converged solve and gradients ------------------------------------------------
    def default_tol(self):
        """Relative residual of the converged solves, 1e-10: the single-precision form
        refreshes its float recurrence with the true residual formed in double, so both
        forms reach the same tolerance."""
        return 1e-10

    def solve(self, b, tol=None, max_iters=20000, stream=None):
        """x = M^-1 b (PCG to a relative preconditioned residual); returns (x, iters, rel)."""
        x = self._new(self.n_coeffs)
        it, rel = ctypes.c_int(0), ctypes.c_double(0.0)
        self._check(self.L.fewha_solve(self.h, self._dev(b, self.n_coeffs, "b"),
                                       self._dev(x, self.n_coeffs, "x"),
                                       self.default_tol() if tol is None else float(tol),
                                       int(max_iters), ctypes.byref(it), ctypes.byref(rel),
                                       _stream(stream)))
        return x, it.value, rel.value

    def reconstruct_converged(self, slopes, tol=None, max_iters=20000, dm_out=None, stream=None):
        """a~ = F W^T M^-1 b(s) (no gain); kept for backward().  Returns (a~, iters, rel)."""
        if dm_out is None:
            dm_out = self._new(self.n_act)
        it, rel = ctypes.c_int(0), ctypes.c_double(0.0)
        self._check(self.L.fewha_reconstruct_converged(
            self.h, self._dev(slopes, self.n_slopes, "slopes"), self._dev(dm_out, self.n_act, "dm_out"),
            self.default_tol() if tol is None else float(tol), int(max_iters), ctypes.byref(it),
            ctypes.byref(rel), _stream(stream)))
        return dm_out, it.value, rel.value

    def fit_ls(self, c, directions, weights, n_fit, eps, tol=None, max_iters=5000, dm_out=None, stream=None):
        """Least-squares DM fit of the layers W^T c over fitting directions ((theta_x,
        theta_y) pairs in rad, with weights), on n_fit + 1 pupil nodes per side with
        Tikhonov weight eps.  Returns (commands, CG iterations, relative residual); the
        default tol is 1e-7 in single and 1e-12 in double precision."""
        if dm_out is None:
            dm_out = self._new(self.n_act)
        if tol is None:
            tol = 1e-7 if self.dtype == torch.float32 else 1e-12
        k = len(directions)
        if len(weights) != k:
            raise ValueError("need one weight per fitting direction")
        tx = (ctypes.c_double * k)(*[float(d[0]) for d in directions])
        ty = (ctypes.c_double * k)(*[float(d[1]) for d in directions])
        w = (ctypes.c_double * len(weights))(*[float(x) for x in weights])
        cfg = LsFit(k, tx, ty, w, int(n_fit), float(eps))
        it, rel = ctypes.c_int(0), ctypes.c_double(0.0)
        self._check(self.L.fewha_fit_ls(self.h, ctypes.byref(cfg), self._dev(c, self.n_coeffs, "c"),
                                        self._dev(dm_out, self.n_act, "dm_out"), float(tol), int(max_iters),
                                        ctypes.byref(it), ctypes.byref(rel), _stream(stream)))
        return dm_out, it.value, rel.value

    def backward(self, grad_dm, stream=None):
        """Gradients (slopes tensor, alpha, per-layer Cn2 weights) of J with dJ/da~ = grad_dm
        at the last converged reconstruction."""
        gs = self._new(self.n_slopes)
        ga = ctypes.c_double(0.0)
        nl = len(self._structs[2])
        gw = (ctypes.c_double * nl)()
        self._check(self.L.fewha_backward(self.h, self._dev(grad_dm, self.n_act, "grad_dm"),
                                          self._dev(gs, self.n_slopes, "grad_slopes"),
                                          ctypes.byref(ga), gw, _stream(stream)))
        return gs, ga.value, list(gw)

    def bench_stage(self, stage, reps, stream=None):
        """Enqueue `reps` launches of one hot-path kernel (timing; clobbers the warm state)."""
        self._check(self.L.fewha_bench_stage(self.h, STAGES[stage], int(reps), _stream(stream)))

    def set_wait_limit(self, polls, extra=0):
        """Polls before a grid-wide wait of the persistent frame gives up; `extra` > 0 makes
        every wait run out (tests of the timeout path)."""
        self._check(self.L.fewha_set_wait_limit(self.h, int(polls), int(extra)))

    def device_bytes(self):
        """Device memory held by the instance, in bytes."""
        n = ctypes.c_int64(0)
        self._check(self.L.fewha_device_bytes(self.h, ctypes.byref(n)))
        return n.value

    def frame_launches(self):
        n = ctypes.c_int(0)
        self._check(self.L.fewha_frame_launches(self.h, ctypes.byref(n)))
        return n.value

    def diagonals(self, stream=None):
        D = self._new(self.n_coeffs)
        J = self._new(self.n_coeffs)
        self._check(self.L.fewha_get_diagonals(self.h, self._dev(D, self.n_coeffs, "D"),
                                               self._dev(J, self.n_coeffs, "J"), _stream(stream)))
        return D, J


def _ptr_array(ts):
    return (_VP * len(ts))(*[ctypes.c_void_p(t.data_ptr()) for t in ts])


class Batch:
    """Many Reconstructor instances (uneven sizes) reconstructing one frame each in one
    graph replay: every step of the frame is one launch over all instances' work items."""

    def __init__(self, recons):
        self.recons = list(recons)          # keeps the members alive
        if not self.recons:
            raise ValueError("empty batch")
        self.L = lib()
        hs = (_VP * len(self.recons))(*[r.h for r in self.recons])
        b = _VP()
        rc = self.L.fewha_batch_create(hs, len(self.recons), ctypes.byref(b))
        if rc != 0:
            raise FewhaError(rc, self.recons[0].L.fewha_last_error(self.recons[0].h).decode())
        self.b = b
        self.dtype = self.recons[0].dtype

    def _check(self, rc):
        if rc != 0:
            raise FewhaError(rc, self.L.fewha_batch_last_error(self.b).decode())

    def _tables(self, slopes, dms):
        if len(slopes) != len(self.recons):
            raise ValueError("one slope vector per instance")
        if dms is None:
            dms = [r._new(r.n_act) for r in self.recons]
        for r, s, d in zip(self.recons, slopes, dms):
            r._dev(s, r.n_slopes, "slopes")
            r._dev(d, r.n_act, "dm_out")
        return dms, _ptr_array(slopes), _ptr_array(dms)

    @property
    def config(self):
        c = BatchConfig()
        self._check(self.L.fewha_batch_get_config(self.b, ctypes.byref(c)))
        return {"order": c.order, "groups": c.groups, "vec_passes": c.vec_passes,
                "pair_threads": c.pair_threads, "proj_taps": c.proj_taps, "vec_threads": c.vec_threads}

    @config.setter
    def config(self, cfg):
        """Launch shape: order, groups, vec_passes and (optional, 0 = default) pair_threads,
        proj_taps, vec_threads (see fewha_batch_config)."""
        c = BatchConfig(cfg["order"], cfg["groups"], cfg["vec_passes"], cfg.get("pair_threads", 0),
                        cfg.get("proj_taps", 0), cfg.get("vec_threads", 0))
        self._check(self.L.fewha_batch_set_config(self.b, ctypes.byref(c)))

    def reconstruct(self, slopes, dm_out=None, stream=None):
        """One frame of every instance (device tensors); returns the DM command tensors."""
        dms, sp, dp = self._tables(slopes, dm_out)
        self._check(self.L.fewha_batch_reconstruct(self.b, sp, dp, _stream(stream)))
        return dms

    def autotune(self, slopes, dm_out=None, reps=10, stream=None):
        """Time every launch configuration on these slopes and keep the fastest; the
        members' warm state is restored.  Returns (config, mean frame time in us)."""
        dms, sp, dp = self._tables(slopes, dm_out)
        us = ctypes.c_float(0.0)
        self._check(self.L.fewha_batch_autotune(self.b, sp, dp, int(reps), ctypes.byref(us),
                                                _stream(stream)))
        return self.config, us.value

    def close(self):
        if getattr(self, "b", None):
            self.L.fewha_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def reconstruct_batched(recons, slopes, dm_out=None, stream=None):
    """fewha_reconstruct_batched: the batched frame through the library's own batch cache."""
    recons = list(recons)
    if dm_out is None:
        dm_out = [r._new(r.n_act) for r in recons]
    for r, s, d in zip(recons, slopes, dm_out):
        r._dev(s, r.n_slopes, "slopes")
        r._dev(d, r.n_act, "dm_out")
    L = lib()
    hs = (_VP * len(recons))(*[r.h for r in recons])
    fn = L.fewha_reconstruct_batched if recons[0].precision == 32 else L.fewha_reconstruct_batched_f64
    rc = fn(hs, len(recons), _ptr_array(slopes), _ptr_array(dm_out), _stream(stream))
    if rc != 0:
        raise FewhaError(rc, L.fewha_last_error(recons[0].h).decode())
    return dm_out

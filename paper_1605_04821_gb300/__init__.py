"""GB300 (sm_103a) solver for HJB equations with the implicit truncated LISL Scheme 2.

Python binding of the C ABI in include/sl_hjb.h (ctypes; argument marshalling only).  Every
step of the solve runs in the library's CUDA kernels; PyTorch provides device memory and
streams.  Importing this package does not need a GPU; loading the library does need the
built libslhjb.so, and any call fails loudly when it is missing.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libslhjb.so")

SL_OK, SL_EINVAL, SL_ENOMEM, SL_ECUDA, SL_ECFL = 0, 1, 2, 3, 4
SL_ENOCONV_PI, SL_ENOCONV_KRYLOV, SL_EBREAKDOWN, SL_ENAN, SL_ETIMEOUT = 5, 6, 7, 8, 9
STATUS_NAMES = {0: "SL_OK", 1: "SL_EINVAL", 2: "SL_ENOMEM", 3: "SL_ECUDA", 4: "SL_ECFL",
                5: "SL_ENOCONV_PI", 6: "SL_ENOCONV_KRYLOV", 7: "SL_EBREAKDOWN", 8: "SL_ENAN",
                9: "SL_ETIMEOUT"}

EXPORTED = ["sl_opts_default", "sl_hjb_create", "sl_hjb_step", "sl_hjb_solve",
            "sl_hjb_last_error", "sl_hjb_destroy", "sl_hjb_improve", "sl_hjb_set_policy",
            "sl_hjb_build_hierarchy", "sl_hjb_apply", "sl_hjb_vcycle", "sl_hjb_linear_solve",
            "sl_hjb_level_info", "sl_hjb_num_levels", "sl_launch_count",
            "sl_hjb_vcycle_noalloc", "sl_hjb_solve_record", "sl_hjb_adjoint", "sl_hjb_reset",
            "sl_batch_create", "sl_batch_run", "sl_batch_worker_of", "sl_batch_plan",
            "sl_batch_last_error", "sl_batch_destroy", "sl_amg_create", "sl_amg_num_levels",
            "sl_amg_level", "sl_amg_apply", "sl_amg_last_error", "sl_amg_destroy",
            "sl_hjb_recorded_policy", "sl_hjb_set_launch", "sl_batch_autotune",
            "sl_hjb_level_stats", "sl_hjb_inject_breakdown"]


class SlGrid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("x_lo", ctypes.c_double),
                ("x_hi", ctypes.c_double), ("y_lo", ctypes.c_double), ("y_hi", ctypes.c_double)]


class SlControls(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int), ("P", ctypes.c_int), ("sigma", ctypes.c_void_p),
                ("b", ctypes.c_void_p), ("c", ctypes.c_void_p), ("sigma_field", ctypes.c_void_p)]


# sl_field_cb: void (*)(double t, const sl_grid *grid, int m, double *dev_out, void *user, void *stream)
FIELD_CB = ctypes.CFUNCTYPE(None, ctypes.c_double, ctypes.POINTER(SlGrid), ctypes.c_int, ctypes.c_void_p,
                            ctypes.c_void_p, ctypes.c_void_p)


class SlSource(ctypes.Structure):
    _fields_ = [("nf", ctypes.c_int), ("nq", ctypes.c_int), ("phi", ctypes.c_void_p),
                ("G_dev", ctypes.c_void_p), ("tau_kind", ctypes.c_void_p),
                ("tau_rate", ctypes.c_void_p), ("npsi", ctypes.c_int), ("Psi_dev", ctypes.c_void_p),
                ("psi_kind", ctypes.c_void_p), ("psi_rate", ctypes.c_void_p),
                ("f_cb", FIELD_CB), ("psi_cb", FIELD_CB), ("cb_user", ctypes.c_void_p)]


class SlOpts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("levels", ctypes.c_int), ("nu1", ctypes.c_int),
                ("nu2", ctypes.c_int), ("omega", ctypes.c_double), ("krylov_tol", ctypes.c_double),
                ("kry_max", ctypes.c_int), ("inner_tol", ctypes.c_double), ("ir_max", ctypes.c_int),
                ("pi_tol", ctypes.c_double), ("pi_max", ctypes.c_int), ("tie_rel", ctypes.c_double),
                ("argmin_screen", ctypes.c_int), ("rebuild_frac", ctypes.c_double),
                ("use_graphs", ctypes.c_int), ("coarse_tail_rows", ctypes.c_int),
                ("extrapolate", ctypes.c_int), ("precond", ctypes.c_int), ("amg_k_levels", ctypes.c_int),
                ("smoother", ctypes.c_int), ("fine_tma", ctypes.c_int),
                ("coarse_fusion", ctypes.c_int), ("howard_init", ctypes.c_int),
                ("howard_loose_tol", ctypes.c_double), ("argmin_skip", ctypes.c_int),
                ("ir_recursive", ctypes.c_int)]


class SlInstance(ctypes.Structure):
    _fields_ = [("grid", SlGrid), ("ctrl", SlControls), ("src", SlSource),
                ("u_dev", ctypes.c_void_p), ("t0", ctypes.c_double), ("T", ctypes.c_double),
                ("n_steps", ctypes.c_int)]


class SlTuneChoice(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("instances", ctypes.c_int), ("coarse_tail_rows", ctypes.c_int),
                ("probe_seconds", ctypes.c_double)]


class SlLevelStats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("reach", ctypes.c_int), ("explicit_rows", ctypes.c_longlong),
                ("class_nnz", ctypes.c_longlong), ("explicit_nnz", ctypes.c_longlong),
                ("explicit_entries", ctypes.c_longlong)]


class SlStats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int), ("pi_iters", ctypes.c_int), ("krylov_iters", ctypes.c_int),
                ("ir_iters", ctypes.c_int), ("rebuilds", ctypes.c_int),
                ("policy_changes", ctypes.c_longlong), ("explicit_rows", ctypes.c_longlong),
                ("res_final", ctypes.c_double), ("t_argmin_ms", ctypes.c_double),
                ("t_hier_ms", ctypes.c_double), ("t_solve_ms", ctypes.c_double),
                ("graph_steps", ctypes.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def load(path: Optional[str] = None) -> ctypes.CDLL:
    """Loads libslhjb.so (build it with paper_1605_04821_gb300.build first)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: run `python -m paper_1605_04821_gb300.build` "
                           "(the solver has no CPU fallback)")
    lib = ctypes.CDLL(path)
    vp, i, d, ll = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
    sig = {
        "sl_opts_default": (None, [ctypes.POINTER(SlOpts)]),
        "sl_hjb_create": (i, [ctypes.POINTER(vp), ctypes.POINTER(SlGrid), ctypes.POINTER(SlControls),
                              ctypes.POINTER(SlSource), ctypes.POINTER(SlOpts), vp]),
        "sl_hjb_step": (i, [vp, vp, d, d, vp, ctypes.POINTER(SlStats), vp]),
        "sl_hjb_solve": (i, [vp, vp, d, d, i, vp, ctypes.POINTER(SlStats), vp]),
        "sl_hjb_last_error": (ctypes.c_char_p, [vp]),
        "sl_hjb_destroy": (None, [vp]),
        "sl_hjb_improve": (i, [vp, vp, d, vp, ctypes.POINTER(ll), vp]),
        "sl_hjb_set_policy": (i, [vp, vp, vp]),
        "sl_hjb_build_hierarchy": (i, [vp, d, vp]),
        "sl_hjb_apply": (i, [vp, i, i, vp, vp, vp]),
        "sl_hjb_vcycle": (i, [vp, i, vp, vp, vp]),
        "sl_hjb_linear_solve": (i, [vp, vp, vp, d, d, ctypes.POINTER(SlStats), vp]),
        "sl_hjb_level_info": (i, [vp, i, ctypes.POINTER(i), ctypes.POINTER(ll), ctypes.POINTER(ll)]),
        "sl_hjb_num_levels": (i, [vp]),
        "sl_hjb_level_stats": (i, [vp, i, ctypes.POINTER(SlLevelStats)]),
        "sl_launch_count": (ll, []),
        "sl_hjb_vcycle_noalloc": (i, [vp, i, vp, vp, vp]),
        "sl_hjb_solve_record": (i, [vp, vp, d, d, i, i, ctypes.POINTER(SlStats), vp]),
        "sl_hjb_adjoint": (i, [vp, vp, vp, vp, i, vp, vp, ctypes.POINTER(SlStats), vp]),
        "sl_hjb_reset": (i, [vp]),
        "sl_hjb_inject_breakdown": (i, [vp, i]),
        "sl_hjb_recorded_policy": (i, [vp, i, vp, vp]),
        "sl_hjb_set_launch": (i, [vp, i, i]),
        "sl_batch_autotune": (i, [vp, i, i, vp, i, ctypes.POINTER(i)]),
        "sl_batch_create": (i, [ctypes.POINTER(vp), i, ctypes.POINTER(SlInstance),
                                ctypes.POINTER(SlOpts), i]),
        "sl_batch_run": (i, [vp, vp, ctypes.POINTER(SlStats)]),
        "sl_batch_worker_of": (i, [vp, i]),
        "sl_batch_plan": (i, [i, vp, i, vp]),
        "sl_batch_last_error": (ctypes.c_char_p, [vp]),
        "sl_batch_destroy": (None, [vp]),
        "sl_amg_create": (i, [ctypes.POINTER(vp), i, vp, vp, vp, ctypes.POINTER(SlOpts)]),
        "sl_amg_num_levels": (i, [vp]),
        "sl_amg_level": (i, [vp, i, ctypes.POINTER(i), ctypes.POINTER(ll), vp, vp, vp, vp]),
        "sl_amg_apply": (i, [vp, i, vp, vp, vp]),
        "sl_amg_last_error": (ctypes.c_char_p, [vp]),
        "sl_amg_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class SLError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def launch_count() -> int:
    """Kernel launches issued by the library since it was loaded."""
    return int(load().sl_launch_count())


def default_opts(**kw) -> SlOpts:
    o = SlOpts()
    load().sl_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _ptr(t) -> int:
    return t.data_ptr()


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class _DeviceView:
    """A device array of n x n FP64 values, as the CUDA array interface describes it (lets
    torch alias library-owned memory without a copy)."""

    def __init__(self, ptr: int, n: int):
        self.__cuda_array_interface__ = {"shape": (n, n), "typestr": "<f8", "data": (ptr, False),
                                         "version": 2, "strides": None}


class FieldCallback:
    """Wraps fn(t, m, out) as an sl_field_cb.  `out` is an (n, n) float64 CUDA tensor aliasing
    the library's buffer; fn runs with the library's stream as torch's current stream, so its
    torch operations are ordered before the kernels that read the values.  An exception inside
    fn cannot cross the C ABI: it is kept and re-raised by the Solver method that triggered it."""

    def __init__(self, fn, n: int):
        self.fn = fn
        self.n = n
        self.error = None

        def _cb(t, grid, m, dev_out, user, stream):
            import torch
            try:
                out = torch.as_tensor(_DeviceView(dev_out, self.n))
                st = torch.cuda.ExternalStream(stream) if stream else torch.cuda.default_stream()
                with torch.cuda.stream(st):
                    self.fn(t, m, out)
            except BaseException as e:  # noqa: BLE001 - kept and re-raised on the Python side
                if self.error is None:
                    self.error = e

        self.c = FIELD_CB(_cb)

    def raise_pending(self):
        if self.error is not None:
            e, self.error = self.error, None
            raise RuntimeError("a coefficient callback raised") from e


def _describe(keep: list, n, lo, hi, sigma, phi, G, tau_kind, tau_rate, Psi=None, psi_kind=None,
              psi_rate=None, b=None, c=None, sigma_field=None, f_cb=None, psi_cb=None):
    """sl_grid / sl_controls / sl_source for one problem.  Host arrays and the device tensors
    are appended to `keep` (which must outlive the structs); the last two entries are G and
    Psi (or None).  f_cb / psi_cb: FieldCallback objects or None (G / Psi are then unused)."""
    import torch

    def host(a, dtype):
        arr = np.ascontiguousarray(a, dtype=dtype)
        keep.append(arr)
        return arr.ctypes.data_as(ctypes.c_void_p)

    if sigma_field is not None:   # x-dependent diffusion shared by all controls
        sigma_field = np.ascontiguousarray(sigma_field, dtype=np.float64)
        assert sigma_field.shape[:3] == (n, n, 2)
        K, P = len(np.atleast_2d(phi)), sigma_field.shape[3]
        sig_ptr, fld_ptr = None, host(sigma_field, np.float64)
    else:
        sigma = np.ascontiguousarray(sigma, dtype=np.float64)
        K, _, P = sigma.shape
        sig_ptr, fld_ptr = host(sigma, np.float64), None
    grid = SlGrid(n, n, lo, hi, lo, hi)
    ctrl = SlControls(K, P, sig_ptr,
                      host(b, np.float64) if b is not None else None,
                      host(c, np.float64) if c is not None else None, fld_ptr)
    if f_cb is None:
        G = G.contiguous()
        assert G.is_cuda and G.dtype == torch.float64 and G.shape[2:] == (n, n)
        nf, nq = G.shape[0], G.shape[1]
        g_ptr = _ptr(G)
    else:
        nf, nq, g_ptr = np.atleast_2d(phi).shape[1], 0, None
        tau_kind, tau_rate = np.zeros(1, dtype=np.int32), np.zeros(1)
    npsi = 0
    psi_ptr = None
    if Psi is not None and psi_cb is None:
        Psi = Psi.contiguous()
        npsi = Psi.shape[0]
        psi_ptr = _ptr(Psi)
    src = SlSource(nf, nq, host(phi, np.float64), g_ptr, host(tau_kind, np.int32),
                   host(tau_rate, np.float64), npsi, psi_ptr,
                   host(psi_kind, np.int32) if npsi else None,
                   host(psi_rate, np.float64) if npsi else None,
                   f_cb.c if f_cb is not None else FIELD_CB(),
                   psi_cb.c if psi_cb is not None else FIELD_CB(), None)
    keep.append(f_cb)
    keep.append(psi_cb)
    keep.append(G)
    keep.append(Psi)
    return grid, ctrl, src


class Solver:
    """Owns one library handle.  All tensors are CUDA tensors on the current device.

    G: (nf, nq, n, n) float64 source tables; Psi: (npsi, n, n) float64 or None.  The handle
    keeps references to G and Psi, which must stay alive and unchanged.
    f_cb / psi_cb: optional coefficient callbacks fn(t, m, out) (sl_field_cb) that write
    F_m(t, .) or psi(t, .) into the (n, n) float64 CUDA tensor `out` at each step's time; they
    replace G (then pass G=None) and Psi.
    """

    def __init__(self, n: int, lo: float, hi: float, sigma: np.ndarray, phi: np.ndarray, G,
                 tau_kind, tau_rate, Psi=None, psi_kind=None, psi_rate=None, b=None, c=None,
                 sigma_field=None, opts: Optional[SlOpts] = None, stream=None, f_cb=None,
                 psi_cb=None, **opt_kw):
        lib = load()
        self._lib = lib
        self._keep = []
        self._cbs = [FieldCallback(fn, n) if fn is not None else None for fn in (f_cb, psi_cb)]
        grid, ctrl, src = _describe(self._keep, n, lo, hi, sigma, phi, G, tau_kind, tau_rate, Psi,
                                    psi_kind, psi_rate, b, c, sigma_field, *self._cbs)
        self.n, self.K, self.P = n, ctrl.K, ctrl.P
        self.general = ctrl.sigma_field is not None
        self._G = self._keep[-2]
        self._Psi = self._keep[-1]
        self.opts = opts if opts is not None else default_opts(**opt_kw)
        h = ctypes.c_void_p()
        st = lib.sl_hjb_create(ctypes.byref(h), ctypes.byref(grid), ctypes.byref(ctrl),
                               ctypes.byref(src), ctypes.byref(self.opts), _stream(stream))
        if st != SL_OK:
            raise SLError(st, "sl_hjb_create failed (see stderr)")
        self.h = h
        self.m = n - 2

    def reset(self):
        """sl_hjb_reset: the next step starts like the first step of a new handle."""
        self._check(self._lib.sl_hjb_reset(self.h))

    def inject_breakdown(self, iterations: int):
        """sl_hjb_inject_breakdown: mark the BiCGSTAB iteration `iterations` from now as a
        breakdown (a test hook for the restart path; 0 cancels)."""
        self._check(self._lib.sl_hjb_inject_breakdown(self.h, iterations))

    def close(self):
        if getattr(self, "h", None):
            self._lib.sl_hjb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        for cb in self._cbs:
            if cb is not None:
                cb.raise_pending()
        if st != SL_OK:
            raise SLError(st, self._lib.sl_hjb_last_error(self.h).decode())

    def step(self, u, t_n: float, dt: float, policy_out=None, stream=None) -> dict:
        s = SlStats()
        self._check(self._lib.sl_hjb_step(self.h, _ptr(u), t_n, dt,
                                          _ptr(policy_out) if policy_out is not None else None,
                                          ctypes.byref(s), _stream(stream)))
        return s.as_dict()

    def solve(self, u, t0: float, T: float, n_steps: int, policy_out=None, stream=None) -> dict:
        s = SlStats()
        self._check(self._lib.sl_hjb_solve(self.h, _ptr(u), t0, T, n_steps,
                                           _ptr(policy_out) if policy_out is not None else None,
                                           ctypes.byref(s), _stream(stream)))
        return s.as_dict()

    def improve(self, x_ext, t: float, policy_out=None, stream=None) -> int:
        ch = ctypes.c_longlong(0)
        self._check(self._lib.sl_hjb_improve(self.h, _ptr(x_ext), t,
                                             _ptr(policy_out) if policy_out is not None else None,
                                             ctypes.byref(ch), _stream(stream)))
        return ch.value

    def set_policy(self, policy, stream=None):
        self._check(self._lib.sl_hjb_set_policy(self.h, _ptr(policy), _stream(stream)))

    def build_hierarchy(self, dt: float, stream=None):
        self._check(self._lib.sl_hjb_build_hierarchy(self.h, dt, _stream(stream)))

    def apply(self, level: int, x, y, stream=None):
        import torch
        prec = 0 if x.dtype == torch.float64 else 1
        self._check(self._lib.sl_hjb_apply(self.h, level, prec, _ptr(x), _ptr(y), _stream(stream)))

    def vcycle(self, b, x, stream=None):
        import torch
        prec = 0 if b.dtype == torch.float64 else 1
        self._check(self._lib.sl_hjb_vcycle(self.h, prec, _ptr(b), _ptr(x), _stream(stream)))

    def vcycle_noalloc(self, b, x, stream=None):
        """sl_hjb_vcycle_noalloc: the V-cycle with the library's static scratch (no allocation)."""
        import torch
        prec = 0 if b.dtype == torch.float64 else 1
        self._check(self._lib.sl_hjb_vcycle_noalloc(self.h, prec, _ptr(b), _ptr(x), _stream(stream)))

    def linear_solve(self, u_prev, x_ext, t: float, dt: float, stream=None) -> dict:
        s = SlStats()
        self._check(self._lib.sl_hjb_linear_solve(self.h, _ptr(u_prev), _ptr(x_ext), t, dt,
                                                  ctypes.byref(s), _stream(stream)))
        return s.as_dict()

    def solve_record(self, u, t0: float, T: float, n_steps: int, ckpt_every: int = 1,
                     stream=None) -> dict:
        """sl_hjb_solve that records policies and checkpoints for a later adjoint()."""
        s = SlStats()
        self._check(self._lib.sl_hjb_solve_record(self.h, _ptr(u), t0, T, n_steps, ckpt_every,
                                                  ctypes.byref(s), _stream(stream)))
        return s.as_dict()

    def adjoint(self, w, dJ_dg, dJ_dG=None, dsigma=None, stream=None):
        """Backward pass of the last solve_record for J = sum w U^N.

        Fills dJ_dg (n, n) and, if given, dJ_dG (nf, nq, n, n); dsigma (nparam, K, 2, P) host
        array of d sigma / d theta_p.  Returns (dJ/dtheta as a numpy array, stats dict).
        """
        s = SlStats()
        np_ = 0
        ds_ptr = None
        out = np.zeros(0)
        if dsigma is not None:
            dsigma = np.ascontiguousarray(dsigma, dtype=np.float64)
            np_ = dsigma.shape[0]
            out = np.zeros(np_)
            ds_ptr = dsigma.ctypes.data_as(ctypes.c_void_p)
        self._check(self._lib.sl_hjb_adjoint(
            self.h, _ptr(w), _ptr(dJ_dg), _ptr(dJ_dG) if dJ_dG is not None else None, np_, ds_ptr,
            out.ctypes.data_as(ctypes.c_void_p) if np_ else None, ctypes.byref(s), _stream(stream)))
        return out, s.as_dict()

    def set_launch(self, use_graphs: int, coarse_tail_rows: int):
        """sl_hjb_set_launch: graph mode and single-block V-cycle tail of this handle."""
        self._check(self._lib.sl_hjb_set_launch(self.h, use_graphs, coarse_tail_rows))
        self.opts.use_graphs = use_graphs
        self.opts.coarse_tail_rows = coarse_tail_rows

    def recorded_policy(self, step: int, policy_out, stream=None):
        """sl_hjb_recorded_policy: the policy of step `step` (1-based) of the last solve_record."""
        self._check(self._lib.sl_hjb_recorded_policy(self.h, step, _ptr(policy_out), _stream(stream)))

    def num_levels(self) -> int:
        return self._lib.sl_hjb_num_levels(self.h)

    def level_info(self, level: int):
        n = ctypes.c_int(0)
        ex = ctypes.c_longlong(0)
        nnz = ctypes.c_longlong(0)
        self._check(self._lib.sl_hjb_level_info(self.h, level, ctypes.byref(n), ctypes.byref(ex),
                                                ctypes.byref(nnz)))
        return n.value, ex.value, nnz.value

    def level_stats(self, level: int) -> dict:
        """sl_hjb_level_stats: reach, class and explicit non-zeros of one hierarchy level."""
        st = SlLevelStats()
        self._check(self._lib.sl_hjb_level_stats(self.h, level, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in st._fields_}


def _problem_args(prob, dev):
    """Positional and keyword arguments of Solver / _describe for a `workloads.Problem`."""
    import torch
    if prob.G is None:
        raise ValueError("the library needs the separable source form (phi, G, tau)")
    G = torch.as_tensor(prob.G, dtype=torch.float64, device=dev)
    psi = prob.psi_fn(0.0)
    kw = {}
    if np.any(psi != 0.0):
        Psi = torch.as_tensor(psi[None], dtype=torch.float64, device=dev)
        kw = dict(Psi=Psi, psi_kind=np.array([0], dtype=np.int32), psi_rate=np.array([0.0]))
    args = (prob.n, prob.lo, prob.hi, prob.sigma, prob.phi, G,
            np.asarray(prob.tau_kind, dtype=np.int32), np.asarray(prob.tau_rate, dtype=np.float64))
    kw.update(b=prob.drift, c=prob.c)
    if prob.sigma_fn is not None:
        # x-dependent sigma: the library takes one field shared by all controls, and constant
        # per-control drifts
        x = prob.lo + prob.h * np.arange(prob.n, dtype=np.float64)
        X1, X2 = np.meshgrid(x, x, indexing="xy")
        field = prob.sigma_fn(0, X1, X2)
        for k in range(1, prob.K):
            if not np.array_equal(prob.sigma_fn(k, X1, X2), field):
                raise ValueError("the library needs sigma(x) shared by all controls")
        kw["sigma_field"] = field
        if prob.drift_fn is not None:
            b = np.stack([prob.drift_fn(k, X1, X2)[0, 0] for k in range(prob.K)])
            for k in range(prob.K):
                if not np.all(prob.drift_fn(k, X1, X2) == b[k]):
                    raise ValueError("the library needs a constant drift per control")
            kw["b"] = b
    return args, kw


def solver_from_problem(prob, device=None, stream=None, **opt_kw) -> Solver:
    """Marshals a `workloads.Problem` with a separable source into a Solver."""
    import torch
    args, kw = _problem_args(prob, device or torch.device("cuda"))
    return Solver(*args, stream=stream, **kw, **opt_kw)


class Batch:
    """sl_batch: independent instances solved concurrently by `workers` host threads, each
    with its own stream.  `problems` are `workloads.Problem`s; `us` are their state tensors
    (n x n float64 on the device: in g, out U(t0 + T)), kept by the batch."""

    def __init__(self, problems, us, workers: int = 8, t0: float = 0.0, device=None, **opt_kw):
        import torch
        lib = load()
        self._lib = lib
        self._keep = []
        dev = device or torch.device("cuda")
        n = len(problems)
        arr = (SlInstance * n)()
        for i, (p, u) in enumerate(zip(problems, us)):
            args, kw = _problem_args(p, dev)
            grid, ctrl, src = _describe(self._keep, *args, **kw)
            assert u.is_cuda and u.dtype == torch.float64 and u.is_contiguous()
            self._keep.append(u)
            arr[i] = SlInstance(grid, ctrl, src, _ptr(u), t0, p.T, p.n_steps)
        self._arr = arr
        self.n = n
        self.opts = default_opts(**opt_kw)
        b = ctypes.c_void_p()
        st = lib.sl_batch_create(ctypes.byref(b), n, arr, ctypes.byref(self.opts), workers)
        if st != SL_OK:
            raise SLError(st, "sl_batch_create failed (see stderr)")
        self.b = b

    def run(self):
        """Solves every instance; returns (statuses, per-instance stats dicts)."""
        st = (ctypes.c_int * self.n)()
        stats = (SlStats * self.n)()
        self._lib.sl_batch_run(self.b, st, stats)
        return [int(x) for x in st], [s.as_dict() for s in stats]

    def autotune(self, probe_steps: int = 3, max_tail_rows: int = 16384):
        """sl_batch_autotune: per grid size, the V-cycle tail that gave the fastest probe run of
        the whole batch; returns [{n, instances, coarse_tail_rows, probe_seconds}, ...]."""
        out = (SlTuneChoice * 64)()
        k = ctypes.c_int(0)
        st = self._lib.sl_batch_autotune(self.b, probe_steps, max_tail_rows, out, 64, ctypes.byref(k))
        if st != SL_OK:
            raise SLError(st, self.last_error())
        return [{f: getattr(out[j], f) for f, _ in SlTuneChoice._fields_} for j in range(min(k.value, 64))]

    def worker_of(self, i: int) -> int:
        return int(self._lib.sl_batch_worker_of(self.b, i))

    def last_error(self) -> str:
        return self._lib.sl_batch_last_error(self.b).decode()

    def close(self):
        if getattr(self, "b", None):
            self._lib.sl_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lpt_plan(costs, bins: int):
    """sl_batch_plan: the LPT assignment (bin of each item) the batch uses."""
    costs = np.ascontiguousarray(costs, dtype=np.float64)
    out = np.zeros(len(costs), dtype=np.int32)
    st = load().sl_batch_plan(len(costs), costs.ctypes.data_as(ctypes.c_void_p), bins,
                              out.ctypes.data_as(ctypes.c_void_p))
    if st != SL_OK:
        raise SLError(st, "sl_batch_plan: bad arguments")
    return out


class Amg:
    """sl_amg: the aggregation hierarchy of a given CSR matrix (scipy.sparse) and its K-cycle."""

    def __init__(self, A, **opt_kw):
        import scipy.sparse as sp
        lib = load()
        self._lib = lib
        A = sp.csr_matrix(A)
        A.sort_indices()
        A.sum_duplicates()
        self.n = A.shape[0]
        rp = np.ascontiguousarray(A.indptr, dtype=np.int32)
        ci = np.ascontiguousarray(A.indices, dtype=np.int32)
        va = np.ascontiguousarray(A.data, dtype=np.float64)
        opts = default_opts(**opt_kw)
        a = ctypes.c_void_p()
        st = lib.sl_amg_create(ctypes.byref(a), self.n, rp.ctypes.data_as(ctypes.c_void_p),
                               ci.ctypes.data_as(ctypes.c_void_p), va.ctypes.data_as(ctypes.c_void_p),
                               ctypes.byref(opts))
        if st != SL_OK:
            raise SLError(st, "sl_amg_create failed (see stderr)")
        self.a = a

    def num_levels(self) -> int:
        return int(self._lib.sl_amg_num_levels(self.a))

    def level(self, l: int):
        """(agg or None, scipy CSR matrix) of level l."""
        import scipy.sparse as sp
        n = ctypes.c_int(0)
        nnz = ctypes.c_longlong(0)
        self._lib.sl_amg_level(self.a, l, ctypes.byref(n), ctypes.byref(nnz), None, None, None, None)
        agg = np.zeros(n.value, dtype=np.int32) if l < self.num_levels() - 1 else None
        rp = np.zeros(n.value + 1, dtype=np.int32)
        ci = np.zeros(nnz.value, dtype=np.int32)
        va = np.zeros(nnz.value, dtype=np.float64)
        st = self._lib.sl_amg_level(self.a, l, ctypes.byref(n), ctypes.byref(nnz),
                                    agg.ctypes.data_as(ctypes.c_void_p) if agg is not None else None,
                                    rp.ctypes.data_as(ctypes.c_void_p), ci.ctypes.data_as(ctypes.c_void_p),
                                    va.ctypes.data_as(ctypes.c_void_p))
        if st != SL_OK:
            raise SLError(st, "sl_amg_level failed")
        return agg, sp.csr_matrix((va, ci, rp), shape=(n.value, n.value))

    def apply(self, b, x, stream=None):
        import torch
        prec = 0 if b.dtype == torch.float64 else 1
        st = self._lib.sl_amg_apply(self.a, prec, _ptr(b), _ptr(x), _stream(stream))
        if st != SL_OK:
            raise SLError(st, self._lib.sl_amg_last_error(self.a).decode())

    def close(self):
        if getattr(self, "a", None):
            self._lib.sl_amg_destroy(self.a)
            self.a = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def instance_cost(prob) -> float:
    """The batch's cost estimate of one instance: nodes x steps x (K + 32)."""
    return float(prob.n) * prob.n * prob.n_steps * (prob.K + 32)


def shard(problems, world: int, rank: int):
    """Indices of the instances that rank `rank` of `world` solves: the LPT plan over ranks
    (instances are independent, so no collective is needed on the data path)."""
    plan = lpt_plan([instance_cost(p) for p in problems], world)
    return [i for i in range(len(problems)) if plan[i] == rank]


def hjb_solve(solver: Solver, g, G, T: float, n_steps: int, ckpt_every: int = 1, theta=None,
              dsigma=None):
    """U(T) = implicit march of `solver` from g, differentiable in g, G and theta.

    G must be the solver's own source tensor (the handle reads it in place).  theta (nparam,)
    names scalar parameters of sigma whose directions d sigma / d theta are `dsigma`
    (nparam, K, 2, P); its value is the point the solver was created at and is not read.
    The backward pass is the library's discrete adjoint (sl_hjb_adjoint).
    """
    import torch

    class _HJBSolve(torch.autograd.Function):
        @staticmethod
        def forward(ctx, g_, G_, theta_):
            if G_.data_ptr() != solver._G.data_ptr():
                raise ValueError("G must be the tensor the solver was created with")
            u = g_.detach().clone().contiguous()
            solver.solve_record(u, 0.0, T, n_steps, ckpt_every)
            return u

        @staticmethod
        def backward(ctx, grad_u):
            w = grad_u.detach().contiguous().to(torch.float64)
            dg = torch.zeros_like(w)
            dG = torch.zeros_like(solver._G) if ctx.needs_input_grad[1] else None
            dth, _ = solver.adjoint(w, dg, dG, dsigma if theta is not None else None)
            gth = None
            if theta is not None:
                gth = torch.as_tensor(dth, dtype=theta.dtype, device=theta.device)
            return dg, dG, gth

    th = theta if theta is not None else torch.zeros(0, dtype=torch.float64, device=g.device)
    return _HJBSolve.apply(g, G, th)

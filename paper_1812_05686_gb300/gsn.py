"""Thin ctypes binding of libgsn (include/gsn.h): argument marshalling only.

Every step of the likelihood runs in the CUDA kernels of libgsn.so; this module
only converts numpy arrays / torch tensors into the pointers and sizes of the C
ABI.  There is no fallback: if the library was not built, load_library()
raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgsn.so")

GSN_OK = 0
GSN_ERR_ARG, GSN_ERR_CUDA, GSN_ERR_NONPOSITIVE_MU, GSN_ERR_NONFINITE, GSN_ERR_STATE, GSN_ERR_NOMEM = -1, -2, -3, -4, -5, -6
GSN_ERR_TIMEOUT = -7
GSN_FP64, GSN_MIXED = 0, 1
GSN_RES_GAUSS, GSN_RES_GAMMA, GSN_RES_GGAMMA = 0, 1, 2
GSN_ANA, GSN_ANA_SHIFT, GSN_ANA_PEAK, GSN_MC_TEMPLATE = 0, 1, 2, 3


class gsn_options(C.Structure):
    _fields_ = [("precision", C.c_int), ("resolution", C.c_int), ("band_cut", C.c_double),
                ("birks_s0", C.c_double), ("birks_s1", C.c_double), ("device", C.c_int),
                ("stream", C.c_void_p), ("max_toys_per_launch", C.c_int), ("use_graphs", C.c_int),
                ("autotune", C.c_int)]


class GsnError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"gsn error {code}: {msg}")
        self.code = code


_lib = None
_DP = C.POINTER(C.c_double)
_IP = C.POINTER(C.c_int)


def load_library(path: str = LIB_PATH):
    """Load libgsn.so once; raises if it has not been built (no CPU fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libgsn.so not found at {path}: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = C.CDLL(path)
    vp = C.c_void_p
    sig = {
        "gsn_default_options": (C.c_int, [C.POINTER(gsn_options)]),
        "gsn_create": (C.c_int, [C.POINTER(vp), C.POINTER(gsn_options)]),
        "gsn_destroy": (None, [vp]),
        "gsn_last_error": (C.c_char_p, [vp]),
        "gsn_n_slots": (C.c_int, [C.c_int]),
        "gsn_set_data": (C.c_int, [vp, C.c_int, _IP, C.POINTER(_DP), C.POINTER(_DP), _DP, _IP, _IP]),
        "gsn_set_species": (C.c_int, [vp, C.c_int, C.c_int, _DP, _DP, _IP, _DP, C.POINTER(C.c_ubyte)]),
        "gsn_set_params": (C.c_int, [vp, C.c_int, _IP, C.c_int, _IP, _DP, _DP]),
        "gsn_eval": (C.c_int, [vp, _DP, _DP]),
        "gsn_eval_grad": (C.c_int, [vp, _DP, _DP, _DP]),
        "gsn_eval_grad_batch": (C.c_int, [vp, C.c_int, _DP, _DP, _IP, _DP, _DP]),
        "gsn_eval_grad_batch_dev": (C.c_int, [vp, C.c_int, vp, vp, vp, vp, vp, vp]),
        "gsn_expected": (C.c_int, [vp, _DP, C.c_int, _DP]),
        "gsn_stream": (vp, [vp]),
        "gsn_profile": (C.c_int, [vp, C.c_int]),
        "gsn_profile_read": (C.c_int, [vp, C.c_int, _DP, C.POINTER(C.c_longlong), C.POINTER(C.c_ulonglong)]),
        "gsn_kernel_name": (C.c_char_p, [C.c_int]),
        "gsn_peak_probe": (C.c_int, [C.c_int, C.c_int, _DP]),
        "gsn_eval_grad_noalloc": (C.c_int, [vp, vp, vp, vp, vp]),
        "gsn_plan_info": (C.c_int, [vp, C.c_int, C.c_int, _IP]),
        "gsn_set_dataset_factors": (C.c_int, [vp, C.c_int, C.c_int, _DP, _DP]),
        "gsn_set_template": (C.c_int, [vp, C.c_int, C.c_int, _DP]),
        "gsn_minimize_batch_dev": (C.c_int, [vp, C.c_int, vp, vp, vp, C.POINTER(C.c_ubyte), _DP, _DP, _DP,
                                             C.c_int, C.c_double, C.c_double, vp, vp, vp]),
        "gsn_set_secondary": (C.c_int, [vp, C.c_int, C.c_int, _IP, C.c_int, _DP, _DP]),
        "gsn_n_counts": (C.c_int, [vp]),
        "gsn_minimize_batch_scaled_dev": (C.c_int, [vp, C.c_int, vp, vp, vp, C.POINTER(C.c_ubyte), _DP, _DP, vp,
                                                    C.c_int, C.c_double, C.c_double, C.c_double, vp, vp, vp]),
        "gsn_window_scales_dev": (C.c_int, [vp, C.c_int, vp, vp, _DP, C.c_double, vp]),
        "gsn_fit_rates_batch_dev": (C.c_int, [vp, C.c_int, vp, vp, vp, C.POINTER(C.c_ubyte), _DP, _DP, C.c_int,
                                              C.c_double, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    """Names the binding expects the library to export (one per declaration of gsn.h)."""
    return ["gsn_default_options", "gsn_create", "gsn_destroy", "gsn_last_error", "gsn_n_slots",
            "gsn_set_data", "gsn_set_species", "gsn_set_params", "gsn_eval", "gsn_eval_grad",
            "gsn_eval_grad_batch", "gsn_eval_grad_batch_dev", "gsn_expected", "gsn_stream",
            "gsn_profile", "gsn_profile_read", "gsn_kernel_name", "gsn_peak_probe", "gsn_eval_grad_noalloc",
            "gsn_plan_info", "gsn_set_dataset_factors", "gsn_set_template", "gsn_minimize_batch_dev",
            "gsn_set_secondary", "gsn_n_counts", "gsn_minimize_batch_scaled_dev", "gsn_window_scales_dev",
            "gsn_fit_rates_batch_dev"]


GSN_K_COUNT = 8
GSN_PROBE_FFMA, GSN_PROBE_EX2, GSN_PROBE_DFMA, GSN_PROBE_NODE, GSN_PROBE_EX2_BIAS = 0, 1, 2, 3, 4


def peak_probe(which, device=0):
    """Operations per second of one instruction class on every SM (gsn_peak_probe)."""
    lib = load_library()
    out = C.c_double()
    rc = lib.gsn_peak_probe(device, which, C.byref(out))
    if rc != GSN_OK:
        raise GsnError(rc, "gsn_peak_probe failed")
    return out.value


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_DP)


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(_IP)


class Context:
    """One gsn_ctx: a problem (data, species, parameter map) on one device and stream."""

    def __init__(self, precision=GSN_FP64, resolution=GSN_RES_GAUSS, band_cut=0.0, device=0, stream=None,
                 birks_s0=1.55, birks_s1=0.155, max_toys_per_launch=0, use_graphs=1, autotune=1):
        self.lib = load_library()
        o = gsn_options()
        self.lib.gsn_default_options(C.byref(o))
        o.precision, o.resolution, o.band_cut = precision, resolution, band_cut
        o.birks_s0, o.birks_s1, o.device = birks_s0, birks_s1, device
        o.stream = stream
        o.max_toys_per_launch = max_toys_per_launch
        o.use_graphs, o.autotune = use_graphs, autotune
        h = C.c_void_p()
        rc = self.lib.gsn_create(C.byref(h), C.byref(o))
        if rc != GSN_OK:
            raise GsnError(rc, "gsn_create failed")
        self.h = h
        self.precision = precision
        self.n_params = 0
        self.total_bins = 0
        self.n_datasets = 0

    def close(self):
        if getattr(self, "h", None):
            self.lib.gsn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != GSN_OK:
            raise GsnError(rc, self.lib.gsn_last_error(self.h).decode())
        return rc

    def last_error(self):
        return self.lib.gsn_last_error(self.h).decode()

    # ---------------------------------------------------------- setup ----
    def set_data(self, edges, counts, exposures, win_lo, win_hi):
        D = len(edges)
        keep = [_d(e) for e in edges] + [_d(c) for c in counts]
        nb = np.array([len(e) - 1 for e in edges], np.int32)
        eptr = (_DP * D)(*[k[1] for k in keep[:D]])
        cptr = (_DP * D)(*[k[1] for k in keep[D:]])
        nb_, nbp = _i(nb)
        ex_, exp_ = _d(exposures)
        lo_, lop = _i(win_lo)
        hi_, hip = _i(win_hi)
        self._check(self.lib.gsn_set_data(self.h, D, nbp, eptr, cptr, exp_, lop, hip))
        self.n_datasets = D
        self.total_bins = int(nb.sum())
        self.n_bins = [int(x) for x in nb]

    def set_species(self, fine_centres, spectra, kind, shift, dataset_mask):
        spectra = np.ascontiguousarray(spectra, np.float64)
        S, K = spectra.shape
        E_, Ep = _d(fine_centres)
        S_, Sp = _d(spectra)
        k_, kp = _i(kind)
        sh_, shp = _d(shift if shift is not None else np.zeros(S))
        m = np.ascontiguousarray(dataset_mask, np.uint8)
        self._check(self.lib.gsn_set_species(self.h, S, K, Ep, Sp, kp, shp, m.ctypes.data_as(C.POINTER(C.c_ubyte))))
        self.n_species = S

    def set_params(self, n_params, slot_map, pull_param=(), pull_centre=(), pull_width=()):
        sm_, smp = _i(np.asarray(slot_map).reshape(-1))
        pp_, ppp = _i(np.asarray(pull_param, np.int32).reshape(-1))
        pc_, pcp = _d(np.asarray(pull_centre, np.float64).reshape(-1))
        pw_, pwp = _d(np.asarray(pull_width, np.float64).reshape(-1))
        self._check(self.lib.gsn_set_params(self.h, n_params, smp, len(pp_), ppp, pcp, pwp))
        self.n_params = n_params

    # ------------------------------------------------------------ calls ----
    def eval(self, params):
        p_, pp = _d(params)
        out = C.c_double()
        rc = self.lib.gsn_eval(self.h, pp, C.byref(out))
        return rc, out.value

    def eval_grad(self, params):
        p_, pp = _d(params)
        out = C.c_double()
        g = np.zeros(self.n_params)
        rc = self.lib.gsn_eval_grad(self.h, pp, C.byref(out), g.ctypes.data_as(_DP))
        return rc, out.value, g

    def eval_grad_batch(self, params, counts, windows, want_grad=True):
        params = np.ascontiguousarray(params, np.float64)
        T = params.shape[0]
        c_, cp = _d(counts)
        w_, wp = _i(windows)
        nll = np.zeros(T)
        g = np.zeros((T, self.n_params)) if want_grad else None
        rc = self.lib.gsn_eval_grad_batch(self.h, T, params.ctypes.data_as(_DP), cp, wp, nll.ctypes.data_as(_DP),
                                          g.ctypes.data_as(_DP) if want_grad else None)
        return rc, nll, g

    def eval_grad_batch_dev(self, params, counts, windows, nll, grad=None, status=None):
        """Device tensors (torch): params (T,P) f64, counts (T,B) f64, windows (T,D,2) i32, nll (T,) f64."""
        T = int(params.shape[0])
        ptr = lambda t: C.c_void_p(t.data_ptr()) if t is not None else None
        return self.lib.gsn_eval_grad_batch_dev(self.h, T, ptr(params), ptr(counts), ptr(windows), ptr(nll),
                                                ptr(grad), ptr(status))

    def expected(self, params, dataset):
        p_, pp = _d(params)
        out = np.zeros((self.n_bins[dataset], self.n_species))
        self._check(self.lib.gsn_expected(self.h, pp, dataset, out.ctypes.data_as(_DP)))
        return out

    def stream(self):
        return self.lib.gsn_stream(self.h)

    def set_dataset_factors(self, resp_scale=None, rate_factor=None):
        """Per-dataset response multipliers (D, 5) and rate fractions (D, S) of a multivariate fit."""
        rs = pr = None
        rf = pf = None
        if resp_scale is not None:
            rs, pr = _d(resp_scale)
        if rate_factor is not None:
            rf, pf = _d(rate_factor)
        self._check(self.lib.gsn_set_dataset_factors(self.h, self.n_datasets, self.n_species, pr, pf))

    def minimize_batch_dev(self, params, counts, wins, free, lo=None, hi=None, scale=None, max_evals=200,
                           gtol=-1.0, ftol=-1.0, nll=None, evals=None, status=None, scale_dev=None, edm=0.0):
        """Batched L-BFGS minimisation (gsn_minimize_batch_dev; with scale_dev, a [T][P] device tensor
        of per-toy scales, gsn_minimize_batch_scaled_dev, which also takes the edm stopping rule);
        params (torch, device) is overwritten with the minima.  Returns (nll, evals, status) device
        tensors."""
        import torch
        T = params.shape[0]
        dev = params.device
        nll = nll if nll is not None else torch.empty(T, dtype=torch.float64, device=dev)
        evals = evals if evals is not None else torch.empty(T, dtype=torch.int32, device=dev)
        status = status if status is not None else torch.empty(T, dtype=torch.int32, device=dev)
        fr = np.ascontiguousarray(np.asarray(free, dtype=np.uint8))
        args = []
        for v in (lo, hi, scale):
            if v is None:
                args.append(None)
            else:
                a, pa = _d(v)
                args.append((a, pa))
        head = (self.h, T, C.c_void_p(params.data_ptr()), C.c_void_p(counts.data_ptr()), C.c_void_p(wins.data_ptr()),
                fr.ctypes.data_as(C.POINTER(C.c_ubyte)), args[0][1] if args[0] else None,
                args[1][1] if args[1] else None)
        outs = (C.c_void_p(nll.data_ptr()), C.c_void_p(evals.data_ptr()), C.c_void_p(status.data_ptr()))
        if scale_dev is not None:
            self._check(self.lib.gsn_minimize_batch_scaled_dev(*head, C.c_void_p(scale_dev.data_ptr()), int(max_evals),
                                                               float(gtol), float(ftol), float(edm), *outs))
        else:
            if edm > 0.0:
                raise ValueError("the edm stopping rule needs per-toy scales (scale_dev)")
            self._check(self.lib.gsn_minimize_batch_dev(*head, args[2][1] if args[2] else None, int(max_evals),
                                                        float(gtol), float(ftol), *outs))
        return nll, evals, status

    def fit_rates_batch_dev(self, params, counts, wins, free, lo=None, hi=None, max_iter=0, tol=0.0):
        """Newton fits over the free rates of every toy (gsn_fit_rates_batch_dev); params (torch,
        device) is overwritten with the minima.  Returns (nll, iters, status) device tensors."""
        import torch
        T = params.shape[0]
        dev = params.device
        nll = torch.empty(T, dtype=torch.float64, device=dev)
        iters = torch.empty(T, dtype=torch.int32, device=dev)
        status = torch.empty(T, dtype=torch.int32, device=dev)
        fr = np.ascontiguousarray(np.asarray(free, dtype=np.uint8))
        lo_ = None if lo is None else _d(lo)
        hi_ = None if hi is None else _d(hi)
        self._check(self.lib.gsn_fit_rates_batch_dev(
            self.h, T, C.c_void_p(params.data_ptr()), C.c_void_p(counts.data_ptr()), C.c_void_p(wins.data_ptr()),
            fr.ctypes.data_as(C.POINTER(C.c_ubyte)), lo_[1] if lo_ else None, hi_[1] if hi_ else None,
            int(max_iter), float(tol), C.c_void_p(nll.data_ptr()), C.c_void_p(iters.data_ptr()),
            C.c_void_p(status.data_ptr())))
        return nll, iters, status

    def window_scales_dev(self, params, wins, scale=None, max_factor=0.0, out=None):
        """Per-toy minimiser scales (gsn_window_scales_dev): a [T][P] device tensor."""
        import torch
        T = params.shape[0]
        out = out if out is not None else torch.empty(T, self.n_params, dtype=torch.float64, device=params.device)
        sc = None if scale is None else _d(scale)
        self._check(self.lib.gsn_window_scales_dev(self.h, T, C.c_void_p(params.data_ptr()),
                                                   C.c_void_p(wins.data_ptr()), sc[1] if sc else None,
                                                   float(max_factor), C.c_void_p(out.data_ptr())))
        return out

    def set_secondary(self, dataset, slice_start, shapes, counts=None):
        """Secondary observable of a dataset: slice boundaries (Q+1,), shapes (S, Q, M), counts (Q, M)."""
        if shapes is None:
            self._check(self.lib.gsn_set_secondary(self.h, int(dataset), 0, None, 0, None, None))
            return
        shapes = np.ascontiguousarray(shapes, np.float64)
        st, pst = _i(np.asarray(slice_start, np.int32))
        sh, psh = _d(shapes)
        Q, M = shapes.shape[1], shapes.shape[2]
        cn = pcn = None
        if counts is not None:
            cn, pcn = _d(np.asarray(counts, np.float64).reshape(-1))
        self._check(self.lib.gsn_set_secondary(self.h, int(dataset), Q, pst, M, psh, pcn))

    def n_counts(self):
        """Values in a toy's counts row (energy bins, then secondary bins)."""
        return self.lib.gsn_n_counts(self.h)

    def set_template(self, species, dataset, hist):
        """Monte Carlo template (visible-bin histogram) of a GSN_MC_TEMPLATE species in one dataset."""
        if hist is None:
            self._check(self.lib.gsn_set_template(self.h, int(species), int(dataset), None))
            return
        h, ph = _d(hist)
        self._check(self.lib.gsn_set_template(self.h, int(species), int(dataset), ph))

    def plan_info(self, n_toys=1, grad=True):
        """Work decomposition of a launch of n_toys toys (gsn_plan_info)."""
        out = (C.c_int * 5)()
        self._check(self.lib.gsn_plan_info(self.h, int(n_toys), int(grad), C.cast(out, _IP)))
        keys = ("nsplit", "bw_warps", "bw_bsplit", "dev_chunks", "tuned")
        return dict(zip(keys, list(out)))

    def profile(self, enable=True):
        self._check(self.lib.gsn_profile(self.h, int(enable)))

    def profile_read(self):
        """{kernel name: (total ms, launches, evaluated (bin, column) pairs)} since the last reset."""
        out = {}
        for k in range(GSN_K_COUNT):
            ms, n, u = C.c_double(), C.c_longlong(), C.c_ulonglong()
            self._check(self.lib.gsn_profile_read(self.h, k, C.byref(ms), C.byref(n), C.byref(u)))
            out[self.lib.gsn_kernel_name(k).decode()] = (ms.value, n.value, u.value)
        return out


def context_from_workload(work: dict, precision=GSN_FP64, counts=None, **kw) -> Context:
    """Configure a Context from a workload dictionary (see inputs.py)."""
    ctx = Context(precision=precision, resolution=int(work["resolution"]),
                  birks_s0=work["birks_s0"], birks_s1=work["birks_s1"], **kw)
    edges = work["edges"]
    sec = work.get("secondary")
    sec_counts = [None] * len(edges)
    if counts is None:
        counts = [np.zeros(len(e) - 1) for e in edges]
    elif not isinstance(counts, (list, tuple)):
        flat = np.asarray(counts, np.float64)
        counts, o = [], 0
        for e in edges:
            counts.append(flat[o:o + len(e) - 1]); o += len(e) - 1
        for d, x in enumerate(sec or []):  # a secondary tail after the energy bins
            if x is not None and flat.size > o:
                n = int(np.prod(np.asarray(x["shapes"]).shape[1:]))
                sec_counts[d] = flat[o:o + n]; o += n
    ctx.set_data(edges, counts, work["exposure"], work["win_lo"], work["win_hi"])
    ctx.set_species(work["fine_centres"], work["spectra"], work["kind"], work["shift"], work["mask"])
    ctx.set_params(int(work["n_params"]), work["slot_map"], work["pull_param"], work["pull_centre"], work["pull_width"])
    if work.get("resp_scale") is not None or work.get("rate_factor") is not None:
        ctx.set_dataset_factors(work.get("resp_scale"), work.get("rate_factor"))
    for s, row in enumerate(work.get("templates") or []):
        for d, hist in enumerate(row or []):
            if hist is not None:
                ctx.set_template(s, d, hist)
    for d, x in enumerate(sec or []):
        if x is not None:
            ctx.set_secondary(d, x["slice_start"], x["shapes"],
                              sec_counts[d] if sec_counts[d] is not None else x.get("counts"))
    return ctx


# --------------------------------------------------------------- autograd ----
def make_autograd():
    """torch.autograd.Function whose forward is gsn_eval_grad and whose backward
    scales the analytic gradient of the adjoint kernel."""
    import torch

    class GsnNLL(torch.autograd.Function):
        @staticmethod
        def forward(fctx, params, ctx):
            rc, nll, g = ctx.eval_grad(params.detach().cpu().double().numpy())
            if rc != GSN_OK:
                raise GsnError(rc, ctx.last_error())
            fctx.save_for_backward(torch.from_numpy(g).to(params.device, params.dtype))
            return torch.tensor(nll, dtype=params.dtype, device=params.device)

        @staticmethod
        def backward(fctx, gout):
            (g,) = fctx.saved_tensors
            return gout * g, None

    return GsnNLL

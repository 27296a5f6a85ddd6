"""Python binding of the C ABI in include/flashmp.h (argument marshalling only).

Every computation runs in libflashmp.so (CUDA, sm_103a). There is no CPU
fallback: if the library is missing or a GPU is not available the calls raise.
Tensors are torch float64 CUDA tensors, contiguous, shaped [3, nz, ny, nx]
(edge / face fields) or [nz, ny, nx] (cell arrays).
"""
from __future__ import annotations

import ctypes as C
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libflashmp.so")

FMP_OK = 0
FMP_ERR_ARG = -1
FMP_ERR_CUDA = -2
FMP_ERR_NOMEM = -3
FMP_ERR_NOT_CONVERGED = -4
FMP_ERR_BREAKDOWN = -5
FMP_ERR_NONFINITE = -6
FMP_ERR_UNSUPPORTED = -7

PRECISIONS = {"fp64": 0, "tf32": 1, "fp16": 2, "bf16": 3, "fp64_ozaki": 4}
KRYLOV = {"fgmres": 0, "bicgstab": 1}


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int)]


class Subdomains(C.Structure):
    _fields_ = [("n_cuts", C.c_int * 3), ("cuts", C.POINTER(C.c_int) * 3), ("overlap", C.c_int)]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int), ("krylov", C.c_int), ("restart", C.c_int), ("rtol", C.c_double),
                ("max_iters", C.c_int), ("use_graph", C.c_int), ("use_learned", C.c_int), ("timing", C.c_int)]


class SolveInfo(C.Structure):
    _fields_ = [("iters", C.c_int), ("restarts", C.c_int), ("true_rel_res", C.c_double),
                ("est_rel_res", C.c_double), ("ms_precond", C.c_float), ("ms_spmv", C.c_float),
                ("ms_orth", C.c_float), ("ms_total", C.c_float), ("used_fallback", C.c_int),
                ("status", C.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class FlashMPError(RuntimeError):
    def __init__(self, status, what):
        super().__init__(f"{what}: {status_string(status)} ({status})")
        self.status = status


_lib = None
_P = C.c_void_p
_D = C.c_double
_I = C.c_int


def lib():
    """Load libflashmp.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with `python -m paper_2508_07193_b300.build`")
    L = C.CDLL(LIB_PATH)
    sig = {
        "fmp_abi_version": (_I, []),
        "fmp_status_string": (C.c_char_p, [_I]),
        "fmp_default_options": (None, [C.POINTER(Options)]),
        "fmp_setup": (_I, [C.POINTER(_P), Grid, _P, _D, C.POINTER(Subdomains), C.POINTER(Options), _P]),
        "fmp_destroy": (None, [_P]),
        "fmp_set_options": (_I, [_P, C.POINTER(Options)]),
        "fmp_set_stream": (_I, [_P, _P]),
        "fmp_get_eps_edge": (_I, [_P, _P]),
        "fmp_get_num_boxes": (_I, [_P, C.POINTER(_I)]),
        "fmp_get_launch_count": (_I, [_P, C.POINTER(C.c_longlong)]),
        "fmp_set_tuning": (_I, [_P, _I, _I]),
        "fmp_get_tuning": (_I, [_P, C.POINTER(_I), C.POINTER(_I)]),
        "fmp_autotune": (_I, [_P, _I, _I, C.POINTER(_I)]),
        "fmp_set_fused": (_I, [_P, _I]),
        "fmp_set_checked": (_I, [_P, _I]),
        "fmp_set_subdomain_form": (_I, [_P, _I]),
        "fmp_get_subdomain_form": (_I, [_P, C.POINTER(_I), C.POINTER(C.c_longlong)]),
        "fmp_get_fused": (_I, [_P, C.POINTER(_I), C.POINTER(_I)]),
        "fmp_set_streamed": (_I, [_P, _I]),
        "fmp_set_orth": (_I, [_P, _I]),
        "fmp_get_orth": (_I, [_P, C.POINTER(_I)]),
        "fmp_get_streamed": (_I, [_P, C.POINTER(_I), C.POINTER(_I)]),
        "fmp_stream_check": (_I, [_P]),
        "fmp_get_box": (_I, [_P, _I, C.POINTER(_I), C.POINTER(_I), C.POINTER(_I), C.POINTER(_I),
                             C.POINTER(_D)]),
        "fmp_curlcurl_apply": (_I, [_P, _P, _P, _D, _D]),
        "fmp_precond_apply": (_I, [_P, _P, _P]),
        "fmp_box_solve": (_I, [_P, _I, _P, _P]),
        "fmp_krylov_solve": (_I, [_P, _P, _P, C.POINTER(SolveInfo)]),
        "fmp_cn_rhs": (_I, [_P, _P, _P, _P, _D, _P]),
        "fmp_h_update": (_I, [_P, _P, _P, _P, _D]),
        "fmp_cn_step": (_I, [_P, _P, _P, _P, _D, C.POINTER(SolveInfo)]),
        "fmp_cn_step_guess": (_I, [_P, _P, _P, _P, _D, _P, C.POINTER(SolveInfo)]),
        "fmp_cnn_num_params": (_I, []),
        "fmp_cnn_set_params": (_I, [_P, _P]),
        "fmp_cnn_get_params": (_I, [_P, _P]),
        "fmp_cnn_apply": (_I, [_P, _P, _P]),
        "fmp_cnn_set_tc": (_I, [_P, _I]),
        "fmp_cnn_add_sample": (_I, [_P, _P, _P]),
        "fmp_cnn_num_samples": (_I, [_P, C.POINTER(_I)]),
        "fmp_cnn_clear_samples": (_I, [_P]),
        "fmp_cnn_grad": (_I, [_P, _I, C.POINTER(_I), _I, _P, C.POINTER(_D)]),
        "fmp_cnn_train": (_I, [_P, _I, _I, C.c_float, C.c_ulonglong, C.POINTER(_D)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def status_string(s):
    return lib().fmp_status_string(int(s)).decode()


def _check(rc, what, ok=(FMP_OK,)):
    if rc not in ok:
        raise FlashMPError(rc, what)
    return rc


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _field(t, shape, name):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous() or tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must be a contiguous float64 CUDA tensor of shape {tuple(shape)}, "
                         f"got {t.dtype} {tuple(t.shape)} on {t.device}")
    return t


def default_options():
    o = Options()
    lib().fmp_default_options(C.byref(o))
    return o


class Context:
    """One grid + material + partition (fmp_setup .. fmp_destroy)."""

    def __init__(self, grid, eps_cell=None, beta=0.25, cuts=None, overlap=0, *, precision="fp64",
                 krylov="fgmres", restart=30, rtol=1e-8, max_iters=1000, timing=False, use_graph=False,
                 use_learned=0, experimental=False, stream=None, device=None):
        L = lib()
        if not torch.cuda.is_available():
            raise RuntimeError("flashmp needs a CUDA device")
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.grid = tuple(int(v) for v in grid)
        nx, ny, nz = self.grid
        self.shape = (3, nz, ny, nx)
        self.beta = float(beta)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        o = self._options(precision, krylov, restart, rtol, max_iters, timing, use_graph, use_learned, experimental)
        sd = None
        self._cut_arrays = None
        if cuts is not None:
            sd = Subdomains()
            arrs = [(C.c_int * len(c))(*[int(v) for v in c]) for c in cuts]
            self._cut_arrays = arrs
            for a in range(3):
                sd.n_cuts[a] = len(cuts[a])
                sd.cuts[a] = C.cast(arrs[a], C.POINTER(C.c_int))
            sd.overlap = int(overlap)
        eps_t = None
        if eps_cell is not None:
            eps_t = torch.as_tensor(eps_cell, dtype=torch.float64).to(self.device).contiguous()
            _field(eps_t, (nz, ny, nx), "eps_cell")
        self._eps_keepalive = eps_t
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            rc = L.fmp_setup(C.byref(h), Grid(nx, ny, nz), _ptr(eps_t), self.beta,
                             C.byref(sd) if sd is not None else None, C.byref(o),
                             C.c_void_p(self.stream.cuda_stream))
        _check(rc, "fmp_setup")
        self._h = h
        self._opts = o

    @staticmethod
    def _options(precision, krylov, restart, rtol, max_iters, timing, use_graph, use_learned=0,
                 experimental=False):
        o = default_options()
        if int(use_learned) >= 2 and not experimental:
            # the in-FGMRES learned correction measured 2.7x the iterations of
            # the plain solver on the dipole runs; it stays for experiments
            raise ValueError("use_learned=2 (learned correction inside FGMRES) is experimental: it measured "
                             "2.7x the iterations of the plain solver; pass experimental=True to use it")
        o.use_learned = int(use_learned)
        o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        o.krylov = KRYLOV[krylov] if isinstance(krylov, str) else int(krylov)
        o.restart = int(restart)
        o.rtol = float(rtol)
        o.max_iters = int(max_iters)
        o.timing = int(bool(timing))
        o.use_graph = int(bool(use_graph))
        return o

    # -- lifetime --------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            lib().fmp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_options(self, **kw):
        cur = dict(precision=self._opts.precision, krylov=self._opts.krylov, restart=self._opts.restart,
                   rtol=self._opts.rtol, max_iters=self._opts.max_iters, timing=self._opts.timing,
                   use_graph=self._opts.use_graph, use_learned=self._opts.use_learned,
                   experimental=self._opts.use_learned >= 2)
        cur.update(kw)
        o = self._options(**cur)
        _check(lib().fmp_set_options(self._h, C.byref(o)), "fmp_set_options")
        self._opts = o

    def set_stream(self, stream):
        _check(lib().fmp_set_stream(self._h, C.c_void_p(stream.cuda_stream)), "fmp_set_stream")
        self.stream = stream

    # -- queries ----------------------------------------------------------
    def empty_field(self):
        return torch.zeros(self.shape, dtype=torch.float64, device=self.device)

    def eps_edge(self):
        out = self.empty_field()
        _check(lib().fmp_get_eps_edge(self._h, _ptr(out)), "fmp_get_eps_edge")
        return out

    def set_tuning(self, slab_group, tile_group):
        _check(lib().fmp_set_tuning(self._h, int(slab_group), int(tile_group)), "fmp_set_tuning")

    def get_tuning(self):
        a, b = C.c_int(), C.c_int()
        _check(lib().fmp_get_tuning(self._h, C.byref(a), C.byref(b)), "fmp_get_tuning")
        return a.value, b.value

    FORMS = {"yee": 0, "compact": 1}

    def set_subdomain_form(self, form):
        """'yee' (Yee boxes with PEC walls, default) or 'compact' (Algorithm 1
        with the Woodbury boundary correction; builds the correction matrices)."""
        f = self.FORMS[form] if isinstance(form, str) else int(form)
        _check(lib().fmp_set_subdomain_form(self._h, f), "fmp_set_subdomain_form")

    def get_subdomain_form(self):
        f, nb = C.c_int(), C.c_longlong()
        _check(lib().fmp_get_subdomain_form(self._h, C.byref(f), C.byref(nb)), "fmp_get_subdomain_form")
        return ("yee", "compact")[f.value], nb.value

    def set_checked(self, on=True):
        """Checked mode: calls raise FlashMPError(FMP_ERR_ARG) on a field with a
        nonzero wall slot (fmp_set_checked)."""
        _check(lib().fmp_set_checked(self._h, int(bool(on))), "fmp_set_checked")

    def set_fused(self, max_extent):
        _check(lib().fmp_set_fused(self._h, int(max_extent)), "fmp_set_fused")

    def get_fused(self):
        a, n = C.c_int(), C.c_int()
        _check(lib().fmp_get_fused(self._h, C.byref(a), C.byref(n)), "fmp_get_fused")
        return a.value, n.value

    def set_streamed(self, mode):
        """bf16 / fp16 boxes outside the fused list: 1 one persistent streamed
        launch (default), 0 the three-pass kernels, 2 a test of its bounded
        waits (fmp_set_streamed)."""
        _check(lib().fmp_set_streamed(self._h, int(mode)), "fmp_set_streamed")

    def get_streamed(self):
        m, n = C.c_int(), C.c_int()
        _check(lib().fmp_get_streamed(self._h, C.byref(m), C.byref(n)), "fmp_get_streamed")
        return m.value, n.value

    ORTH_MODES = {"float64": 0, "fixed": 1, "split": 2}

    def set_orth(self, mode="fixed"):
        """Gram-Schmidt arithmetic of FGMRES (fmp_set_orth): "float64",
        "fixed" (exact fixed-point products on kept copies) or "split" (the
        default: fixed-point products for the oldest vectors of each pass,
        float64 FMAs for the rest); True / False stand for "fixed" /
        "float64", and 0, 1, 2 for the three."""
        if isinstance(mode, bool):
            mode = int(mode)
        elif isinstance(mode, str):
            mode = self.ORTH_MODES[mode]
        _check(lib().fmp_set_orth(self._h, int(mode)), "fmp_set_orth")

    def get_orth(self):
        """The Gram-Schmidt mode as its number: 0 float64, 1 fixed, 2 split."""
        v = C.c_int()
        _check(lib().fmp_get_orth(self._h, C.byref(v)), "fmp_get_orth")
        return v.value

    def stream_check(self):
        """FMP_OK, or FMP_ERR_CUDA when a wait of the streamed solve ran out
        since the last check (returned, not raised; fmp_stream_check)."""
        return lib().fmp_stream_check(self._h)

    def autotune(self, precision="bf16", reps=5, cache=None):
        """Pick the fastest fused setting and work-list grouping for
        `precision` (fmp_autotune), cached in the JSON file `cache` keyed by
        GPU name, grid, partition and precision. Returns (slab group, tile
        group, microseconds per apply, fused max extent)."""
        import json
        key = None
        if cache:
            name = torch.cuda.get_device_name(self.device)
            key = f"{name}|{self.grid}|{self.num_boxes()}|{self.box(0)['m']}|{precision}"
            try:
                with open(cache) as f:
                    table = json.load(f)
            except (OSError, ValueError):
                table = {}
            if key in table and len(table[key]) == 4:
                self.set_tuning(*table[key][:2])
                self.set_fused(table[key][3])
                return tuple(table[key])
        res = (C.c_int * 4)()
        p = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        _check(lib().fmp_autotune(self._h, p, int(reps), res), "fmp_autotune")
        out = (res[0], res[1], res[2], res[3])
        if cache:
            try:
                with open(cache) as f:
                    table = json.load(f)
            except (OSError, ValueError):
                table = {}
            table[key] = list(out)
            with open(cache, "w") as f:
                json.dump(table, f, indent=1)
        return out

    def launch_count(self):
        n = C.c_longlong()
        _check(lib().fmp_get_launch_count(self._h, C.byref(n)), "fmp_get_launch_count")
        return n.value

    def num_boxes(self):
        n = C.c_int()
        _check(lib().fmp_get_num_boxes(self._h, C.byref(n)), "fmp_get_num_boxes")
        return n.value

    def box(self, i):
        a, m, o, n = (C.c_int * 3)(), (C.c_int * 3)(), (C.c_int * 3)(), (C.c_int * 3)()
        e = C.c_double()
        _check(lib().fmp_get_box(self._h, int(i), a, m, o, n, C.byref(e)), "fmp_get_box")
        return dict(ext_lo=tuple(a), m=tuple(m), own_lo=tuple(o), own_n=tuple(n), eps_bar=e.value)

    # -- compute ----------------------------------------------------------
    def curlcurl_apply(self, x, y=None, c_eps=1.0, c_k=None):
        _field(x, self.shape, "x")
        y = self.empty_field() if y is None else _field(y, self.shape, "y")
        c_k = self.beta if c_k is None else c_k
        _check(lib().fmp_curlcurl_apply(self._h, _ptr(x), _ptr(y), float(c_eps), float(c_k)), "fmp_curlcurl_apply")
        return y

    def precond_apply(self, r, z=None):
        _field(r, self.shape, "r")
        z = self.empty_field() if z is None else _field(z, self.shape, "z")
        _check(lib().fmp_precond_apply(self._h, _ptr(r), _ptr(z)), "fmp_precond_apply")
        return z

    def box_solve(self, i, r, x=None):
        mx, my, mz = self.box(i)["m"]
        shp = (3, mz, my, mx)
        _field(r, shp, "r")
        x = torch.zeros(shp, dtype=torch.float64, device=self.device) if x is None else _field(x, shp, "x")
        _check(lib().fmp_box_solve(self._h, int(i), _ptr(r), _ptr(x)), "fmp_box_solve")
        return x

    def krylov_solve(self, b, x=None, check=True):
        _field(b, self.shape, "b")
        x = self.empty_field() if x is None else _field(x, self.shape, "x")
        info = SolveInfo()
        rc = lib().fmp_krylov_solve(self._h, _ptr(b), _ptr(x), C.byref(info))
        if check:
            _check(rc, "fmp_krylov_solve")
        return x, info.as_dict()

    def cn_rhs(self, E, H, J, dt, R=None):
        _field(E, self.shape, "E"); _field(H, self.shape, "H")
        if J is not None:
            _field(J, self.shape, "J")
        R = self.empty_field() if R is None else _field(R, self.shape, "R")
        _check(lib().fmp_cn_rhs(self._h, _ptr(E), _ptr(H), _ptr(J), float(dt), _ptr(R)), "fmp_cn_rhs")
        return R

    def h_update(self, H, E_new, E_old, dt):
        for t, n in ((H, "H"), (E_new, "E_new"), (E_old, "E_old")):
            _field(t, self.shape, n)
        _check(lib().fmp_h_update(self._h, _ptr(H), _ptr(E_new), _ptr(E_old), float(dt)), "fmp_h_update")
        return H

    def cn_step(self, E, H, J, dt, check=True, E_prev=None):
        """One CN step; with E_prev (E^(n-1)) the solve starts from 2 E - E_prev
        (fmp_cn_step_guess)."""
        _field(E, self.shape, "E"); _field(H, self.shape, "H")
        if J is not None:
            _field(J, self.shape, "J")
        info = SolveInfo()
        if E_prev is not None:
            _field(E_prev, self.shape, "E_prev")
            rc = lib().fmp_cn_step_guess(self._h, _ptr(E), _ptr(H), _ptr(J), float(dt), _ptr(E_prev),
                                         C.byref(info))
        else:
            rc = lib().fmp_cn_step(self._h, _ptr(E), _ptr(H), _ptr(J), float(dt), C.byref(info))
        if check:
            _check(rc, "fmp_cn_step")
        return info.as_dict()

    # -- learned component --------------------------------------------------
    def cnn_num_params(self):
        return lib().fmp_cnn_num_params()

    def cnn_set_params(self, params):
        import numpy as np
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.size != self.cnn_num_params():
            raise ValueError(f"expected {self.cnn_num_params()} parameters, got {p.size}")
        _check(lib().fmp_cnn_set_params(self._h, p.ctypes.data_as(C.c_void_p)), "fmp_cnn_set_params")

    def cnn_get_params(self):
        import numpy as np
        p = np.empty(self.cnn_num_params(), dtype=np.float32)
        _check(lib().fmp_cnn_get_params(self._h, p.ctypes.data_as(C.c_void_p)), "fmp_cnn_get_params")
        return p

    def cnn_apply(self, r, out=None):
        _field(r, self.shape, "r")
        out = self.empty_field() if out is None else _field(out, self.shape, "out")
        _check(lib().fmp_cnn_apply(self._h, _ptr(r), _ptr(out)), "fmp_cnn_apply")
        return out

    def cnn_set_tc(self, on=True):
        """Full-volume convolutions on tcgen05 (True, default) or mma.sync
        (False); 2 tests the tcgen05 kernels' bounded waits (fmp_cnn_set_tc)."""
        mode = on if isinstance(on, int) and not isinstance(on, bool) else (1 if on else 0)
        _check(lib().fmp_cnn_set_tc(self._h, mode), "fmp_cnn_set_tc")

    def cnn_add_sample(self, r, e):
        _field(r, self.shape, "r"); _field(e, self.shape, "e")
        _check(lib().fmp_cnn_add_sample(self._h, _ptr(r), _ptr(e)), "fmp_cnn_add_sample")

    def cnn_num_samples(self):
        n = C.c_int()
        _check(lib().fmp_cnn_num_samples(self._h, C.byref(n)), "fmp_cnn_num_samples")
        return n.value

    def cnn_clear_samples(self):
        _check(lib().fmp_cnn_clear_samples(self._h), "fmp_cnn_clear_samples")

    def cnn_grad(self, sample, lo, crop):
        import numpy as np
        g = np.empty(self.cnn_num_params(), dtype=np.float32)
        loss = C.c_double()
        lo_a = (C.c_int * 3)(*[int(v) for v in lo])
        _check(lib().fmp_cnn_grad(self._h, int(sample), lo_a, int(crop), g.ctypes.data_as(C.c_void_p),
                                  C.byref(loss)), "fmp_cnn_grad")
        return loss.value, g

    def cnn_train(self, steps, crop, lr=1e-3, seed=0):
        loss = C.c_double()
        _check(lib().fmp_cnn_train(self._h, int(steps), int(crop), float(lr), int(seed), C.byref(loss)),
               "fmp_cnn_train")
        return loss.value

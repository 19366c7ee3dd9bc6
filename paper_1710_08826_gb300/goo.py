"""Thin ctypes binding of libgoo.so (include/goo.h).

Argument marshalling only: model specs become goo_node arrays, numpy arrays and torch
tensors become column pointers, precision names become GOO_F64/GOO_F32.  Every step of
the likelihood runs in the library's CUDA kernels; there is no CPU fallback -- importing
this module fails if libgoo.so has not been built.
"""
import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_PKG, "libgoo.so")

GOO_OK, GOO_ERR_ARG, GOO_ERR_RANGE, GOO_ERR_CUDA, GOO_ERR_OOM = 0, -1, -2, -3, -4
GOO_ERR_NONPOSITIVE_PDF, GOO_ERR_TIMEOUT, GOO_ERR_STATE, GOO_ERR_UNSUPPORTED = -5, -6, -7, -8
GOO_FIT_ALLOC_FAILED, GOO_FIT_CANCELLED = 6, 7
GOO_F64, GOO_F32 = 0, 1
GOO_LINESHAPE_CACHED, GOO_LINESHAPE_FLOATING = 0, 1
GOO_COEF_CARTESIAN, GOO_COEF_POLAR = 0, 1
GOO_COPY, GOO_BORROW_DEVICE, GOO_COPY_MAPPED, GOO_BORROW_HOST = 0, 1, 2, 3
OP = dict(gauss=1, expo=2, poly2=3, argus=4, prod=10, add=11, bw=20, nr=21, coherent=22, td4=23, amp4=24, td3=25)
ANG = dict(SS=0, VS0=1, SV0=2, VV0=3, VVpar=4, VVperp=5, TS0=6, TV0=7)
NORM = dict(analytic=0, grid=1, mc=2)
MAX_CHILD = 16
PAIR_INDEX = {"12": 0, "13": 1, "23": 2}


class GooNode(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("obs", ctypes.c_int32 * 2), ("par", ctypes.c_int32 * 8),
                ("n_child", ctypes.c_int32), ("child", ctypes.c_int32 * MAX_CHILD),
                ("ival", ctypes.c_int32 * 2), ("dval", ctypes.c_double * 6)]


class GooNormSpec(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("bins", ctypes.c_int32 * 4), ("mc", ctypes.c_void_p)]


class GooFitOptions(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("gradient", ctypes.c_int32), ("max_iter", ctypes.c_int32),
                ("polish", ctypes.c_int32), ("edm_tol", ctypes.c_double), ("refine", ctypes.c_int32)]


class GooFitResult(ctypes.Structure):
    _fields_ = [("nll", ctypes.c_double), ("edm", ctypes.c_double), ("wall_ms", ctypes.c_double),
                ("iterations", ctypes.c_int32), ("nll_evals", ctypes.c_int32), ("grad_evals", ctypes.c_int32),
                ("status", ctypes.c_int32)]


class GooEnvelope(ctypes.Structure):
    _fields_ = [("n12", ctypes.c_int32), ("n13", ctypes.c_int32), ("bound", ctypes.POINTER(ctypes.c_float))]


class GooServerOptions(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_int64), ("max_fits", ctypes.c_int32), ("tile_events", ctypes.c_int32),
                ("max_iter", ctypes.c_int32), ("pad", ctypes.c_int32), ("edm_tol", ctypes.c_double),
                ("envelope", ctypes.c_void_p)]


def _envelope(env):
    """(pointer or None, keep-alive) for an envelope given as None or (n12, n13, bounds)."""
    if env is None:
        return None, None
    n12, n13, bound = env
    b = np.ascontiguousarray(np.asarray(bound, dtype=np.float32).reshape(-1))
    if b.size != int(n12) * int(n13):
        raise ValueError("envelope: n12 * n13 bounds needed")
    e = GooEnvelope(int(n12), int(n13), b.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
    return ctypes.pointer(e), (e, b)


class GooError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"goo error {code}: {msg}")
        self.code = code


def _load():
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"{_LIB_PATH} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'` (needs nvcc)")
    lib = ctypes.CDLL(_LIB_PATH)
    # double* arguments are declared void*: they take ctypes pointers, byref() and arrays as
    # before, and also a numpy array's address as a plain int (the per-evaluation calls)
    vp, dp, i64 = ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64
    sig = {
        "goo_init": (ctypes.c_int, [ctypes.c_int, vp, ctypes.POINTER(vp)]),
        "goo_finalize": (ctypes.c_int, [vp]),
        "goo_last_error": (ctypes.c_char_p, []),
        "goo_version": (ctypes.c_char_p, []),
        "goo_launch_count": (i64, [vp]),
        "goo_timing_enable": (ctypes.c_int, [vp, ctypes.c_int]),
        "goo_timing_read": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_char_p, ctypes.POINTER(i64), dp, ctypes.c_int]),
        "goo_set_wait_limit": (ctypes.c_int, [vp, i64]),
        "goo_debug_withhold_tile": (ctypes.c_int, [vp, i64]),
        "goo_peak_fma": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int, dp, dp]),
        "goo_dataset_upload": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(vp), ctypes.c_int, i64, dp, dp,
                                              ctypes.c_int, ctypes.POINTER(vp), ctypes.POINTER(i64)]),
        "goo_dataset_free": (ctypes.c_int, [vp]),
        "goo_dataset_size": (i64, [vp]),
        "goo_dataset_column": (vp, [vp, ctypes.c_int, ctypes.c_int]),
        "goo_dataset_set_weights": (ctypes.c_int, [vp, dp]),
        "goo_dataset_update": (ctypes.c_int, [vp, ctypes.POINTER(vp), ctypes.c_int, i64, ctypes.c_int,
                                              ctypes.POINTER(i64)]),
        "goo_model_build": (ctypes.c_int, [vp, ctypes.POINTER(GooNode), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           dp, dp, ctypes.POINTER(vp)]),
        "goo_model_set_norm": (ctypes.c_int, [vp, ctypes.POINTER(GooNormSpec)]),
        "goo_model_free": (ctypes.c_int, [vp]),
        "goo_model_components": (ctypes.c_int, [vp]),
        "goo_normalise": (ctypes.c_int, [vp, dp, ctypes.c_int, dp]),
        "goo_nll": (ctypes.c_int, [vp, vp, dp, ctypes.c_int, dp]),
        "goo_nll_grad": (ctypes.c_int, [vp, vp, dp, ctypes.c_int, dp, dp]),
        "goo_eval_logf": (ctypes.c_int, [vp, vp, dp, ctypes.c_int, vp]),
        "goo_nll_partial": (ctypes.c_int, [vp, vp, i64, i64, dp, ctypes.c_int, ctypes.c_int, dp]),
        "goo_nll_grad_streamed": (ctypes.c_int, [vp, vp, ctypes.POINTER(vp), i64, ctypes.c_int, dp, dp, dp,
                                                 ctypes.POINTER(i64)]),
        "goo_combine_partials": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, dp, dp]),
        "goo_gram": (ctypes.c_int, [vp, dp, ctypes.c_int, dp, ctypes.POINTER(ctypes.c_int)]),
        "goo_server_create": (ctypes.c_int, [vp, dp, ctypes.POINTER(ctypes.c_int), dp, ctypes.POINTER(GooServerOptions),
                                             ctypes.POINTER(vp)]),
        "goo_server_submit": (ctypes.c_int, [vp, i64, ctypes.c_uint64, dp, ctypes.POINTER(i64)]),
        "goo_server_step": (ctypes.c_int, [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_int)]),
        "goo_server_result": (ctypes.c_int, [vp, i64, dp, dp, ctypes.c_void_p]),
        "goo_server_stats": (ctypes.c_int, [vp, dp]),
        "goo_server_finished": (ctypes.c_int, [vp, ctypes.POINTER(i64), ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
        "goo_server_cancel": (ctypes.c_int, [vp, i64]),
        "goo_server_fail_allocation": (ctypes.c_int, [vp, i64]),
        "goo_server_free": (ctypes.c_int, [vp]),
        "goo_toy_generate": (ctypes.c_int, [vp, dp, vp, ctypes.c_uint64, i64,
                                            ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)]),
        "goo_toys_generate": (ctypes.c_int, [vp, dp, vp, ctypes.c_int, ctypes.POINTER(ctypes.c_uint64),
                                             ctypes.POINTER(i64), ctypes.POINTER(ctypes.c_float),
                                             ctypes.POINTER(ctypes.c_float)]),
        "goo_nll_grad_batch": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(vp), dp, ctypes.c_int, dp, dp]),
        "goo_fit": (ctypes.c_int, [vp, vp, dp, ctypes.POINTER(ctypes.c_int), dp, ctypes.POINTER(GooFitOptions), dp,
                                   ctypes.POINTER(GooFitResult)]),
        "goo_amplitude_cache": (ctypes.c_int, [vp, vp, dp, ctypes.c_int, ctypes.POINTER(vp),
                                               ctypes.POINTER(ctypes.c_int)]),
        "goo_faddeeva": (ctypes.c_int, [ctypes.c_double, ctypes.c_double, ctypes.c_int, dp]),
        "goo_model_set_lineshapes": (ctypes.c_int, [vp, ctypes.c_int]),
        "goo_model_set_coefficients": (ctypes.c_int, [vp, ctypes.c_int]),
        "goo_model_set_jit": (ctypes.c_int, [vp, ctypes.c_int]),
        "goo_model_jit_status": (ctypes.c_int, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = _load()


def _check(rc):
    if rc != GOO_OK:
        raise GooError(rc, lib.goo_last_error().decode(errors="replace"))
    return rc


def _dbuf(values, n=None):
    a = np.ascontiguousarray(values, dtype=np.float64)
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


_PRECISION = {"f64": GOO_F64, "fp64": GOO_F64, "float64": GOO_F64,
              "f32": GOO_F32, "fp32": GOO_F32, "float32": GOO_F32, "mixed": GOO_F32}


def precision_code(precision):
    if precision in (GOO_F64, GOO_F32):
        return precision
    return _PRECISION[precision]


class Context:
    """A device and a CUDA stream; every call of the library on this context is ordered on it."""

    def __init__(self, device=0, stream=None):
        h = ctypes.c_void_p()
        _check(lib.goo_init(int(device), ctypes.c_void_p(stream) if stream else None, ctypes.byref(h)))
        self.handle = h
        self.device = device

    @property
    def launches(self):
        return int(lib.goo_launch_count(self.handle))

    def timing(self, on=True):
        _check(lib.goo_timing_enable(self.handle, int(bool(on))))

    def set_wait_limit(self, cycles=0):
        """Limit of the kernels' waits for staged input tiles, in SM clocks (0: the default)."""
        _check(lib.goo_set_wait_limit(self.handle, int(cycles)))

    def withhold_tile(self, tile=-1):
        """Failure-detection test hook: the first block of the staged kernels skips the copies of
        its tile number `tile` (-1: off), so that their waits run out."""
        _check(lib.goo_debug_withhold_tile(self.handle, int(tile)))

    def peak_fma(self, kind="f64", iters=None):
        """Measured FMA rate of one pipe ("f64", "f32", "f32x2"): (FMAs per second, launch ms)."""
        code = {"f64": 0, "f32": 1, "f32x2": 2}[kind]
        if iters is None:
            iters = {"f64": 256, "f32": 8192, "f32x2": 4096}[kind]
        rate, ms = ctypes.c_double(), ctypes.c_double()
        _check(lib.goo_peak_fma(self.handle, code, int(iters), ctypes.byref(rate), ctypes.byref(ms)))
        return rate.value, ms.value

    def kernel_times(self, reset=True):
        """{kernel name: (launches, total ms)} recorded since the last reset."""
        cap = 64
        names = ctypes.create_string_buffer(64 * cap)
        counts = (ctypes.c_int64 * cap)()
        ms = (ctypes.c_double * cap)()
        n = lib.goo_timing_read(self.handle, cap, names, counts, ms, int(bool(reset)))
        if n < 0:
            _check(n)
        out = {}
        for i in range(min(n, cap)):
            nm = names.raw[64 * i:64 * (i + 1)].split(b"\0", 1)[0].decode()
            out[nm] = (int(counts[i]), float(ms[i]))
        return out

    def close(self):
        if self.handle:
            _check(lib.goo_finalize(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Dataset:
    """Structure-of-arrays event columns on the device (goo_dataset_upload)."""

    def __init__(self, ctx, columns, lo, hi, dtype="f64", mapped=False, borrow_host=False):
        """columns: host arrays (copied), CUDA tensors (borrowed), with mapped=True pinned
        host tensors / arrays that the ingest kernel reads directly (GOO_COPY_MAPPED), or with
        borrow_host=True pinned float32 host tensors kept by reference and read over the host
        link by every evaluation (GOO_BORROW_HOST)."""
        self.ctx = ctx
        cols = list(columns)
        ncols = len(cols)
        dt = precision_code(dtype)
        self._keep = []
        ptrs = (ctypes.c_void_p * ncols)()
        if borrow_host and (mapped or dt != GOO_F32):
            raise ValueError("borrow_host takes float32 columns (dtype='f32') and excludes mapped")
        flags = GOO_BORROW_HOST if borrow_host else GOO_COPY_MAPPED if mapped else GOO_COPY
        n = None
        for i, c in enumerate(cols):
            if hasattr(c, "is_cuda") and c.is_cuda:
                if mapped:
                    raise ValueError("mapped upload takes pinned host columns, not CUDA tensors")
                flags = GOO_BORROW_DEVICE
                want = "float64" if dt == GOO_F64 else "float32"
                if str(c.dtype) != "torch." + want or not c.is_contiguous():
                    raise ValueError(f"borrowed column {i} must be a contiguous torch.{want} tensor")
                self._keep.append(c)
                ptrs[i] = c.data_ptr()
                size = c.numel()
            else:
                a = np.ascontiguousarray(c, dtype=np.float64 if dt == GOO_F64 else np.float32)
                self._keep.append(a)
                ptrs[i] = a.ctypes.data
                size = a.size
            if n is None:
                n = size
            elif size != n:
                raise ValueError("columns differ in length")
        lo_a, lo_p = _dbuf(lo, ncols)
        hi_a, hi_p = _dbuf(hi, ncols)
        h = ctypes.c_void_p()
        nbad = ctypes.c_int64(0)
        rc = lib.goo_dataset_upload(ctx.handle, ncols, ptrs, dt, int(n or 0), lo_p, hi_p, flags, ctypes.byref(h),
                                    ctypes.byref(nbad))
        self.n_bad = int(nbad.value)
        _check(rc)
        if flags not in (GOO_BORROW_DEVICE, GOO_BORROW_HOST):
            self._keep = []
        self.handle = h
        self.dtype = dtype
        self.n = int(n or 0)
        self.ncols = ncols
        self.lo, self.hi = list(lo_a), list(hi_a)

    @classmethod
    def from_spec(cls, ctx, spec, cols, dtype="f64"):
        names = [o[0] for o in spec["observables"]]
        return cls(ctx, [cols[n] for n in names], [o[1] for o in spec["observables"]],
                   [o[2] for o in spec["observables"]], dtype)

    def column_ptr(self, col, dtype="f64"):
        return lib.goo_dataset_column(self.handle, col, precision_code(dtype))

    def update(self, columns, mapped=False):
        """New events into the same device buffers (goo_dataset_update): host arrays, or with
        mapped=True pinned host columns read by the ingest kernel."""
        cols = list(columns)
        if len(cols) != self.ncols:
            raise ValueError(f"expected {self.ncols} columns")
        dt = precision_code(self.dtype)
        ptrs = (ctypes.c_void_p * self.ncols)()
        keep, n = [], None
        for i, c in enumerate(cols):
            if hasattr(c, "data_ptr"):
                want = "float64" if dt == GOO_F64 else "float32"
                if c.is_cuda or str(c.dtype) != "torch." + want or not c.is_contiguous():
                    raise ValueError(f"column {i} must be a contiguous host torch.{want} tensor")
                ptrs[i] = c.data_ptr()
                size = c.numel()
            else:
                a = np.ascontiguousarray(c, dtype=np.float64 if dt == GOO_F64 else np.float32)
                keep.append(a)
                ptrs[i] = a.ctypes.data
                size = a.size
            if n is None:
                n = size
            elif size != n:
                raise ValueError("columns differ in length")
        nbad = ctypes.c_int64(0)
        rc = lib.goo_dataset_update(self.handle, ptrs, dt, int(n or 0), GOO_COPY_MAPPED if mapped else GOO_COPY,
                                    ctypes.byref(nbad))
        self.n_bad = int(nbad.value)
        if rc == 0 or rc == GOO_ERR_RANGE:
            self.n = 0 if rc else int(n or 0)
        _check(rc)

    def set_weights(self, weights):
        """Per-event weights (a binned dataset: bin centres with their counts), copied to the
        device (goo_dataset_set_weights); None removes them."""
        if weights is None:
            _check(lib.goo_dataset_set_weights(self.handle, None))
            return
        w = np.ascontiguousarray(weights, dtype=np.float64)
        if w.shape != (self.n,):
            raise ValueError(f"weights must have shape ({self.n},)")
        _check(lib.goo_dataset_set_weights(self.handle, w.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))

    def close(self):
        if getattr(self, "handle", None):
            _check(lib.goo_dataset_free(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def spec_to_nodes(spec):
    """Post-order goo_node array for a model spec (see synth/specs.py for the format)."""
    pidx = {p[0]: i for i, p in enumerate(spec["params"])}
    oidx = {o[0]: i for i, o in enumerate(spec["observables"])}
    nodes = []

    def new():
        n = GooNode()
        for j in range(2):
            n.obs[j] = -1
        for j in range(8):
            n.par[j] = -1
        return n

    def emit(node):
        op = node[0]
        n = None
        if op in ("gauss", "expo", "poly2", "argus"):
            n = new()
            n.op = OP[op]
            n.obs[0] = oidx[node[1]]
            for j, name in enumerate(node[2:]):
                n.par[j] = pidx[name]
        elif op == "prod":
            kids = [emit(c) for c in node[1]]
            n = new()
            n.op = OP["prod"]
            n.n_child = len(kids)
            for j, k in enumerate(kids):
                n.child[j] = k
        elif op == "add":
            kids = [emit(c) for c in node[2]]
            n = new()
            n.op = OP["add"]
            n.n_child = len(kids)
            for j, k in enumerate(kids):
                n.child[j] = k
            for j, name in enumerate(node[1]):
                n.par[j] = pidx[name]
        elif op in ("coherent", "td3"):
            kin, amps = node[1], node[2]
            kids = []
            for a in amps:
                m = new()
                m.obs[0], m.obs[1] = oidx["s12"], oidx["s13"]
                if a[0] == "bw":
                    _, pair, spin, m0, w, re, im = a
                    m.op = OP["bw"]
                    m.par[0], m.par[1], m.par[2], m.par[3] = pidx[m0], pidx[w], pidx[re], pidx[im]
                    m.ival[0], m.ival[1] = int(spin), PAIR_INDEX[pair]
                elif a[0] == "nr":
                    m.op = OP["nr"]
                    m.par[2], m.par[3] = pidx[a[1]], pidx[a[2]]
                else:
                    raise ValueError(a[0])
                nodes.append(m)
                kids.append(len(nodes) - 1)
            n = new()
            n.op = OP[op]
            n.obs[0], n.obs[1] = oidx["s12"], oidx["s13"]
            if op == "td3":   # decay-time column and x, y, tau, sigma_t
                n.ival[0] = oidx["t"]
                for j, name in enumerate(node[3]):
                    n.par[j] = pidx[name]
            n.n_child = len(kids)
            for j, k in enumerate(kids):
                n.child[j] = k
            for j, key in enumerate(["M", "m1", "m2", "m3", "r_res", "r_par"]):
                n.dval[j] = float(kin[key])
        elif op == "td4":
            kin, amps, tpar = node[1], node[2], node[3]
            kids = []
            for ang, (m0a, ga), (m0b, gb), re, im, (cre, cim) in amps:
                m = new()
                m.op = OP["amp4"]
                m.ival[0] = ANG[ang]
                m.par[0], m.par[1] = pidx[re], pidx[im]
                for j, v in enumerate((m0a, ga, m0b, gb, cre, cim)):
                    m.dval[j] = float(v)
                nodes.append(m)
                kids.append(len(nodes) - 1)
            n = new()
            n.op = OP["td4"]
            n.n_child = len(kids)
            for j, k in enumerate(kids):
                n.child[j] = k
            for j, name in enumerate(tpar):
                n.par[j] = pidx[name]
            for j, key in enumerate(["M", "m1", "m2", "m3", "m4", "r_res"]):
                n.dval[j] = float(kin[key])
        else:
            raise ValueError(f"unknown node {op}")
        nodes.append(n)
        return len(nodes) - 1

    emit(spec["pdf"])
    arr = (GooNode * len(nodes))(*nodes)
    return arr, len(nodes)


class Model:
    """A compiled model (goo_model_build + goo_model_set_norm)."""

    def __init__(self, ctx, spec, mc=None, norm=None):
        self.ctx = ctx
        self.spec = spec
        self.n_params = len(spec["params"])
        nodes, nn = spec_to_nodes(spec)
        lo_a, lo_p = _dbuf([o[1] for o in spec["observables"]])
        hi_a, hi_p = _dbuf([o[2] for o in spec["observables"]])
        h = ctypes.c_void_p()
        _check(lib.goo_model_build(ctx.handle, nodes, nn, self.n_params, len(spec["observables"]), lo_p, hi_p,
                                   ctypes.byref(h)))
        self.handle = h
        # per-model argument and result buffers of the evaluation calls, with their addresses
        # taken once (a Model is used from one thread at a time)
        self._tb = np.zeros(self.n_params)
        self._ob = np.zeros(3 + self.n_params)
        self._gb = np.zeros(self.n_params)
        self._nb = ctypes.c_double()
        self._tb_a, self._ob_a, self._gb_a = self._tb.ctypes.data, self._ob.ctypes.data, self._gb.ctypes.data
        self._nb_ref = ctypes.byref(self._nb)
        self.mc = mc
        self.set_norm(norm or spec["norm"], mc)
        if spec.get("coef") == "polar":   # (magnitude, phase) coefficient parameters
            _check(lib.goo_model_set_coefficients(self.handle, GOO_COEF_POLAR))

    def set_norm(self, norm, mc=None):
        ns = GooNormSpec()
        ns.kind = NORM[norm[0]]
        if norm[0] == "grid":
            for j, b in enumerate(norm[1]):
                ns.bins[j] = int(b)
        if norm[0] == "mc":
            if mc is None:
                raise ValueError("MC normalisation needs the phase-space Dataset")
            ns.mc = mc.handle
            self.mc = mc
        _check(lib.goo_model_set_norm(self.handle, ctypes.byref(ns)))

    @property
    def n_components(self):
        return int(lib.goo_model_components(self.handle))

    def _theta(self, theta):
        return _dbuf(theta, self.n_params)

    def _theta_addr(self, theta):
        # theta copied into the model's buffer; its address
        if len(theta) != self.n_params:
            raise ValueError(f"expected {self.n_params} values, got {len(theta)}")
        self._tb[:] = theta
        return self._tb_a

    def normalise(self, theta, precision="f64"):
        t, tp = self._theta(theta)
        out = np.zeros(max(self.n_components, 1))
        _check(lib.goo_normalise(self.handle, tp, precision_code(precision),
                                 out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        return out

    def nll(self, ds, theta, precision="f64"):
        tp = self._theta_addr(theta)
        _check(lib.goo_nll(self.handle, ds.handle, tp, precision_code(precision), self._nb_ref))
        return self._nb.value

    def nll_grad(self, ds, theta, precision="f64"):
        tp = self._theta_addr(theta)
        _check(lib.goo_nll_grad(self.handle, ds.handle, tp, precision_code(precision), self._nb_ref, self._gb_a))
        return self._nb.value, self._gb.copy()

    def nll_grad_streamed(self, ds, host_columns, theta, n_chunks=8):
        """FP32 NLL and gradient of pinned float32 host columns (torch tensors made with
        pin_memory()), refilling ds chunk by chunk while earlier chunks are evaluated
        (goo_nll_grad_streamed)."""
        t, tp = self._theta(theta)
        ptrs = (ctypes.c_void_p * len(host_columns))(*[int(c.data_ptr()) for c in host_columns])
        n = int(host_columns[0].numel())
        out = ctypes.c_double()
        g = np.zeros(self.n_params)
        nbad = ctypes.c_int64()
        rc = lib.goo_nll_grad_streamed(self.handle, ds.handle, ptrs, n, int(n_chunks), tp, ctypes.byref(out),
                                       g.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(nbad))
        ds.n = int(lib.goo_dataset_size(ds.handle))
        _check(rc)
        return out.value, g

    def eval_logf(self, ds, theta, precision="f64"):
        import torch
        t, tp = self._theta(theta)
        out = torch.empty(ds.n, dtype=torch.float64, device=f"cuda:{self.ctx.device}")
        _check(lib.goo_eval_logf(self.handle, ds.handle, tp, precision_code(precision),
                                 ctypes.c_void_p(out.data_ptr())))
        return out

    def nll_partial(self, ds, begin, end, theta, precision="f64", want_grad=True):
        tp = self._theta_addr(theta)
        _check(lib.goo_nll_partial(self.handle, ds.handle, int(begin), int(end), tp, precision_code(precision),
                                   int(bool(want_grad)), self._ob_a))
        return self._ob.copy()

    def fit(self, ds, theta0, free=None, scale=None, precision="f32", gradient="adjoint", max_iter=500,
            edm_tol=1e-6, polish=True, errors=True, refine=True):
        """Minimise the NLL (goo_fit).  Returns (theta_hat, errors, info dict)."""
        th, thp = _dbuf(np.array(theta0, dtype=np.float64, copy=True), self.n_params)
        if free is None:
            free = [not p[2] for p in self.spec["params"]]
        if scale is None:
            scale = [p[3] if p[3] > 0 else 1.0 for p in self.spec["params"]]
        fm = (ctypes.c_int * self.n_params)(*[int(bool(v)) for v in free])
        sc, scp = _dbuf(scale, self.n_params)
        opt = GooFitOptions(precision_code(precision), {"adjoint": 0, "fd": 1}[gradient], int(max_iter),
                            int(bool(polish)), float(edm_tol), int(bool(refine)))
        err = np.zeros(self.n_params)
        res = GooFitResult()
        _check(lib.goo_fit(self.handle, ds.handle, thp, fm, scp, ctypes.byref(opt),
                           err.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if errors else None,
                           ctypes.byref(res)))
        info = {k: getattr(res, k) for k, _ in GooFitResult._fields_}
        return th.copy(), err, info

    def set_jit(self, on):
        """Run-time specialisation of the FP32 event kernel for this model (goo_model_set_jit):
        True (default) compiles the kernel for the model's leaf signature on first use, False
        keeps the library's interpreter."""
        _check(lib.goo_model_set_jit(self.handle, 1 if on else 0))

    @property
    def jit_status(self):
        """0 off, 1 on and unused, 2 the last FP32 evaluation ran the specialised kernel, -1
        compilation failed (the interpreter ran)."""
        return int(lib.goo_model_jit_status(self.handle))

    def set_lineshapes(self, mode):
        """'cached' (default: masses and widths are constants of the amplitude cache, their
        gradient entries are 0) or 'floating' (amplitudes and their lineshape derivatives
        evaluated per event and per MC point on every call; full gradient)."""
        code = {"cached": GOO_LINESHAPE_CACHED, "floating": GOO_LINESHAPE_FLOATING}[mode]
        _check(lib.goo_model_set_lineshapes(self.handle, code))

    def gram(self, theta, precision="f64"):
        """MC Gram matrix G_kl (complex K x K, resonances in tree order then the NR amplitude)."""
        t, tp = self._theta(theta)
        out = np.zeros(2 * 16 * 16)
        K = ctypes.c_int()
        _check(lib.goo_gram(self.handle, tp, precision_code(precision),
                            out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(K)))
        k = K.value
        g = out[:2 * k * k].reshape(k, k, 2)
        return g[..., 0] + 1j * g[..., 1]

    def amplitudes(self, ds, theta, precision="f64"):
        """Cached resonance amplitudes of ds as a complex [n_events, n_res] numpy array."""
        import torch
        t, tp = self._theta(theta)
        ptr = ctypes.c_void_p()
        nres = ctypes.c_int()
        _check(lib.goo_amplitude_cache(self.handle, ds.handle, tp, precision_code(precision), ctypes.byref(ptr),
                                       ctypes.byref(nres)))
        n, k = ds.n, nres.value
        if precision_code(precision) == GOO_F32:
            planes = (k + 1) // 2
            buf = torch.empty(planes * n * 4, dtype=torch.float32, device=f"cuda:{self.ctx.device}")
            nbytes = buf.numel() * 4
        else:
            buf = torch.empty(k * n * 2, dtype=torch.float64, device=f"cuda:{self.ctx.device}")
            nbytes = buf.numel() * 8
        torch.cuda.synchronize()
        cudart = ctypes.CDLL("libcudart.so.13")
        rc = cudart.cudaMemcpy(ctypes.c_void_p(buf.data_ptr()), ptr, ctypes.c_size_t(nbytes), 3)
        if rc != 0:
            raise GooError(GOO_ERR_CUDA, f"cudaMemcpy failed ({rc})")
        a = buf.cpu().numpy()
        if precision_code(precision) == GOO_F32:
            a = a.reshape(planes, n, 4)
            out = np.empty((n, k), dtype=np.complex128)
            for j in range(k):
                plane, half = divmod(j, 2)
                out[:, j] = a[plane, :, 2 * half] + 1j * a[plane, :, 2 * half + 1]
            return out
        a = a.reshape(k, n, 2)
        return (a[..., 0] + 1j * a[..., 1]).T

    def close(self):
        if getattr(self, "handle", None):
            _check(lib.goo_model_free(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def toy_generate(model, theta, envelope, seed, n):
    """One toy from the device generator: (s12, s13) float32 arrays.  envelope: None (the
    library's default, computed at theta) or (n12, n13, per-cell bounds)."""
    t, tp = _dbuf(theta, model.n_params)
    a = np.zeros(n, dtype=np.float32)
    b = np.zeros(n, dtype=np.float32)
    ep, keep = _envelope(envelope)
    _check(lib.goo_toy_generate(model.handle, tp, ctypes.cast(ep, ctypes.c_void_p) if ep else None, int(seed), int(n),
                                a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                b.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
    return a, b


def toys_generate(model, theta, envelope, seeds, sizes):
    """Several toys generated together: list of (s12, s13) float32 arrays."""
    t, tp = _dbuf(theta, model.n_params)
    ep, keep = _envelope(envelope)
    k = len(seeds)
    sd = (ctypes.c_uint64 * k)(*[int(v) for v in seeds])
    nn = (ctypes.c_int64 * k)(*[int(v) for v in sizes])
    tot = int(sum(int(v) for v in sizes))
    a = np.zeros(tot, dtype=np.float32)
    b = np.zeros(tot, dtype=np.float32)
    _check(lib.goo_toys_generate(model.handle, tp, ctypes.cast(ep, ctypes.c_void_p) if ep else None, k, sd, nn,
                                 a.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                 b.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
    out, off = [], 0
    for v in sizes:
        out.append((a[off:off + int(v)], b[off:off + int(v)]))
        off += int(v)
    return out


def nll_grad_batch(model, datasets, thetas, precision="f32"):
    """NLL and gradient of several (dataset, theta) pairs in one launch."""
    F = len(datasets)
    th = np.ascontiguousarray(np.asarray(thetas, dtype=np.float64).reshape(F, model.n_params))
    handles = (ctypes.c_void_p * F)(*[d.handle.value for d in datasets])
    nll = np.zeros(F)
    g = np.zeros((F, model.n_params))
    _check(lib.goo_nll_grad_batch(model.handle, F, handles, th.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                  precision_code(precision), nll.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                  g.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return nll, g


class Server:
    """Continuous-batching toy-MC fit server (goo_server_*)."""

    def __init__(self, model, theta_gen, free=None, scale=None, budget_bytes=0, max_fits=0, tile_events=0,
                 max_iter=0, edm_tol=0.0, envelope=None):
        self.model = model
        P = model.n_params
        if free is None:
            free = [not p[2] for p in model.spec["params"]]
        if scale is None:
            scale = [p[3] if p[3] > 0 else 1.0 for p in model.spec["params"]]
        tg, tgp = _dbuf(theta_gen, P)
        fm = (ctypes.c_int * P)(*[int(bool(v)) for v in free])
        sc, scp = _dbuf(scale, P)
        ep, self._env_keep = _envelope(envelope)
        o = GooServerOptions(int(budget_bytes), int(max_fits), int(tile_events), int(max_iter), 0, float(edm_tol),
                             ctypes.cast(ep, ctypes.c_void_p) if ep else None)
        h = ctypes.c_void_p()
        _check(lib.goo_server_create(model.handle, tgp, fm, scp, ctypes.byref(o), ctypes.byref(h)))
        self.handle = h

    def submit(self, n_events, seed, theta_start=None):
        t = ctypes.c_int64()
        if theta_start is None:
            tp = None
        else:
            ts, tp = _dbuf(theta_start, self.model.n_params)
            self._keep = ts
        _check(lib.goo_server_submit(self.handle, int(n_events), int(seed), tp, ctypes.byref(t)))
        return t.value

    def step(self):
        q, a, d = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib.goo_server_step(self.handle, ctypes.byref(q), ctypes.byref(a), ctypes.byref(d)))
        return q.value, a.value, d.value

    def result(self, ticket):
        P = self.model.n_params
        th = np.zeros(P)
        err = np.zeros(P)
        res = GooFitResult()
        rc = lib.goo_server_result(self.handle, int(ticket), th.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                   err.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(res))
        if rc == GOO_ERR_STATE:
            return None
        _check(rc)
        return th, err, {k: getattr(res, k) for k, _ in GooFitResult._fields_}

    def finished(self, cap=1024):
        """Tickets of the fits that finished since the previous call, oldest first."""
        buf = (ctypes.c_int64 * cap)()
        out = []
        while True:
            k = ctypes.c_int()
            _check(lib.goo_server_finished(self.handle, buf, cap, ctypes.byref(k)))
            out.extend(buf[:k.value])
            if k.value < cap:
                return out

    def cancel(self, ticket):
        """End a queued or active fit; its result then has status GOO_FIT_CANCELLED."""
        _check(lib.goo_server_cancel(self.handle, int(ticket)))

    def fail_allocation(self, ticket):
        """Test hook: the admission of this queued fit fails (status GOO_FIT_ALLOC_FAILED)."""
        _check(lib.goo_server_fail_allocation(self.handle, int(ticket)))

    def stats(self):
        out = np.zeros(9)
        _check(lib.goo_server_stats(self.handle, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
        keys = ["rounds", "eval_ms", "gen_ms", "candidates", "accepted", "bound_max", "arena_bytes", "arena_used",
                "envelope_violations"]
        return dict(zip(keys, out.tolist()))

    def close(self):
        if getattr(self, "handle", None):
            _check(lib.goo_server_free(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def combine_partials(parts, n_params):
    """Compensated, index-ordered sum of shard records (goo_combine_partials)."""
    p = np.ascontiguousarray(parts, dtype=np.float64).reshape(-1, 3 + n_params)
    out = np.zeros(3 + n_params)
    _check(lib.goo_combine_partials(p.shape[0], n_params, p.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                    out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return out


def version():
    return lib.goo_version().decode()


def faddeeva(z, precision="f64"):
    """The library's Faddeeva approximation w(z), Im z >= 0, evaluated on the host."""
    out = np.zeros(2)
    _check(lib.goo_faddeeva(float(np.real(z)), float(np.imag(z)), precision_code(precision),
                            out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return complex(out[0], out[1])

"""ctypes binding of libalto (the C ABI in ``include/alto.h``).

Argument marshalling only: every step of format generation, MTTKRP and
CP-ALS runs in the library's CUDA kernels.  PyTorch supplies device memory
and the current stream.  When ``libalto.so`` has not been built the binding
raises instead of falling back to anything else.
"""
import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libalto.so")

ALTO_OK, ALTO_EINVAL, ALTO_ENOMEM, ALTO_ECUDA, ALTO_ETIMEOUT, ALTO_EOVERFLOW, ALTO_ENOTSPD, ALTO_ERANGE = range(8)
STATUS_NAMES = {0: "ALTO_OK", 1: "ALTO_EINVAL", 2: "ALTO_ENOMEM", 3: "ALTO_ECUDA", 4: "ALTO_ETIMEOUT",
                5: "ALTO_EOVERFLOW", 6: "ALTO_ENOTSPD", 7: "ALTO_ERANGE"}
F64, F32, BF16 = 0, 1, 2
VAR_AUTO, VAR_ATOMIC, VAR_WARPAGG, VAR_SMEM, VAR_TEMP, VAR_GENERIC = range(6)
VARIANT_NAMES = {0: "auto", 1: "atomic", 2: "warpagg", 3: "smem", 4: "temp", 5: "generic"}
MAX_MODES = 8

_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class Options(ctypes.Structure):
    _fields_ = [("key_bits", ctypes.c_int), ("nparts", ctypes.c_int64),
                ("variant", ctypes.c_int * MAX_MODES), ("use_flags", ctypes.c_int),
                ("alloc", _ALLOC_FN), ("free", _FREE_FN), ("ctx", ctypes.c_void_p)]


class AltoError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


_lib = None


def lib():
    """Load libalto.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libalto.so is not built (%s); call "
                               "paper_2102_10245_gb300.build.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        P, I, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
        sig = {
            "alto_options_init": [P],
            "alto_create": [P, I, P, I64, P, I, P, I, P, P],
            "alto_mttkrp": [P, I, P, I, I, P, P],
            "alto_cpals": [P, I, I, P, I, P, P, P],
            "alto_get_layout": [P, P, P, P, P, P, P],
            "alto_get_hot_rows": [P, I, P, P],
            "alto_get_stats": [P, P, P, P, P, P, P],
            "alto_export": [P, P, P, P, P, P],
            "alto_transpose": [P, I, P, P, P, P, I, P, P],
            "alto_gram": [P, I64, I, I, I, P, P],
            "alto_set_gram_engine": [P, I],
            "alto_set_variant": [P, I, I],
            "alto_set_parts": [P, I, I64],
            "alto_get_key_bytes": [P, P],
            "alto_resolve_variant": [P, I, I, I, I, P],
            "alto_check": [P, P],
            "alto_destroy": [P],
            "alto_layout_for_dims": [I, P, I, P, P, P, P],
            "alto_decode_host": [I, P, I, I64, P, P],
            "alto_profile": [P, I],
            "alto_profile_read": [P, P, P],
            "alto_launch_count": [P],
            "alto_linearize_noalloc": [I, P, I64, P, I, P, P, P],
            "alto_batch_create": [P, I, P, P, P, P, I, P, P, P],
            "alto_batch_run": [P, P],
            "alto_batch_info": [P, P, P, P, P],
            "alto_batch_destroy": [P],
            "alto_get_mode_stats": [P, I, P, I],
            "alto_get_unit_fit": [P, I, ctypes.c_uint64, P],
            "alto_nn_linear_forward": [P, P, P, P, I, I, I, I, P],
            "alto_nn_linear_backward": [P, P, P, P, P, P, P, P, I, I, I, I, P],
            "alto_nn_mse": [P, P, P, P, I64, ctypes.c_double, P, P],
            "alto_nn_adam": [P, P, P, P, I64, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, I, P],
        }
        for name, args in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = ctypes.c_int
        L.alto_last_error.argtypes = []
        L.alto_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def _check(status):
    if status != ALTO_OK:
        raise AltoError(status, lib().alto_last_error().decode(errors="replace"))


def _stream(stream):
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _dims(dims):
    return (ctypes.c_uint64 * len(dims))(*[int(d) for d in dims])


def _fdtype(t):
    if t.dtype == torch.float64:
        return F64
    if t.dtype == torch.float32:
        return F32
    if t.dtype == torch.bfloat16:
        return BF16
    raise TypeError("factor dtype %s not supported" % t.dtype)


GRAM_AUTO, GRAM_CUDA_CORES, GRAM_TENSOR_CORES = 0, 1, 2


def gram(U, engine=GRAM_AUTO, out=None, stream=None):
    """G = U^T U (R x R, float64, on U's device) of a contiguous CUDA factor
    U (I x R, float64 / float32 / bfloat16); synchronises the stream."""
    if not U.is_cuda or not U.is_contiguous() or U.dim() != 2:
        raise ValueError("U must be a contiguous 2-D CUDA tensor")
    I, R = int(U.shape[0]), int(U.shape[1])
    if out is None:
        out = torch.empty((R, R), dtype=torch.float64, device=U.device)
    _check(lib().alto_gram(ctypes.c_void_p(U.data_ptr()), I, R, _fdtype(U), int(engine),
                           ctypes.c_void_p(out.data_ptr()), _stream(stream)))
    return out


def layout_for_dims(dims, key_bits=0):
    """Host-side layout: (bits_per_mode, masks (N x 2 uint64 words), key_words, total_bits)."""
    N = len(dims)
    bits = (ctypes.c_int * N)()
    masks = (ctypes.c_uint64 * (2 * N))()
    kw = ctypes.c_int()
    tb = ctypes.c_int()
    _check(lib().alto_layout_for_dims(N, _dims(dims), key_bits, bits, masks, ctypes.byref(kw),
                                      ctypes.byref(tb)))
    return list(bits), [(masks[2 * n], masks[2 * n + 1]) for n in range(N)], kw.value, tb.value


def decode_host(dims, keys, key_bits=0):
    """Host de-linearization of a (count, key_words) uint64 numpy array."""
    import numpy as np
    _, _, kw, _ = layout_for_dims(dims, key_bits)
    k = np.ascontiguousarray(keys, dtype=np.uint64).reshape(-1, kw)
    out = np.zeros((k.shape[0], len(dims)), dtype=np.uint32)
    _check(lib().alto_decode_host(len(dims), _dims(dims), key_bits, k.shape[0],
                                  k.ctypes.data_as(ctypes.c_void_p), out.ctypes.data_as(ctypes.c_void_p)))
    return out


def launch_count():
    """Kernels libalto has launched in this process so far."""
    c = ctypes.c_uint64()
    _check(lib().alto_launch_count(ctypes.byref(c)))
    return c.value


def torch_allocator():
    """(alloc, free) callbacks that route libalto allocations through
    PyTorch's caching allocator on the current device and stream."""
    live = {}

    def _alloc(nbytes, ctx):
        try:
            p = torch.cuda.caching_allocator_alloc(int(nbytes))
        except RuntimeError:
            return None
        live[p] = nbytes
        return p

    def _free(ptr, ctx):
        if ptr:
            live.pop(ptr, None)
            torch.cuda.caching_allocator_delete(ptr)
    return _alloc, _free


class Batch:
    """Many MTTKRPs captured as one CUDA graph (alto_batch_create).

    items: list of (AltoTensor, mode, factors (list of device tensors),
    out (device tensor)); all factors share one dtype.  variants: optional
    per-item variant list."""

    def __init__(self, items, variants=None, stream=None):
        n = len(items)
        self._items = items  # keep the tensors alive while the graph exists
        fd = None
        handles = (ctypes.c_void_p * max(n, 1))()
        modes = (ctypes.c_int * max(n, 1))()
        ranks = (ctypes.c_int * max(n, 1))()
        outs = (ctypes.c_void_p * max(n, 1))()
        fptrs = (ctypes.c_void_p * max(n, 1))()
        self._fptr_arrays = []
        for i, (at, mode, factors, out) in enumerate(items):
            handles[i] = at._h.value
            modes[i] = mode
            ref = next(f for m, f in enumerate(factors) if f is not None and (m != mode or at.N == 1))
            ranks[i] = int(ref.shape[1])
            fd = _fdtype(ref) if fd is None else fd
            arr = (ctypes.c_void_p * at.N)(*[(f.data_ptr() if f is not None else 0) for f in factors])
            self._fptr_arrays.append(arr)
            fptrs[i] = ctypes.cast(arr, ctypes.c_void_p).value
            outs[i] = out.data_ptr()
        var = None
        if variants is not None:
            var = (ctypes.c_int * max(n, 1))(*[int(v) for v in variants])
        h = ctypes.c_void_p()
        self._h = None
        _check(lib().alto_batch_create(ctypes.byref(h), n, handles, modes, fptrs, ranks,
                                       fd if fd is not None else F32, outs, var, _stream(stream)))
        self._h = h

    def run(self, stream=None):
        _check(lib().alto_batch_run(self._h, _stream(stream)))

    def info(self):
        a, g, s, k = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(lib().alto_batch_info(self._h, ctypes.byref(a), ctypes.byref(g), ctypes.byref(s), ctypes.byref(k)))
        return dict(items=a.value, groups=g.value, single=s.value, kernels=k.value)

    def close(self):
        if getattr(self, "_h", None):
            lib().alto_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class AltoTensor:
    """An ALTO tensor owned by libalto (Sec. 3 of the paper)."""

    def __init__(self, dims, idx, vals, key_bits=0, nparts=0, variants=None, use_flags=True,
                 allocator=None, stream=None):
        N = len(dims)
        if len(idx) != N:
            raise ValueError("need one index array per mode")
        self.dims = tuple(int(d) for d in dims)
        self.N = N
        M = int(vals.shape[0])
        widths = {torch.int32: 4, torch.uint32: 4, torch.int64: 8}
        idx_bytes = widths[idx[0].dtype] if N else 4
        for a in idx:
            if a.dtype not in widths or widths[a.dtype] != idx_bytes or a.shape[0] != M:
                raise ValueError("index arrays must share one integer width and length nnz")
            if not a.is_contiguous():
                raise ValueError("index arrays must be contiguous")
        if vals.dtype not in (torch.float32, torch.float64, torch.bfloat16) or not vals.is_contiguous():
            raise ValueError("values must be contiguous float32, float64 or bfloat16")
        self.vdtype = {torch.float64: F64, torch.float32: F32, torch.bfloat16: BF16}[vals.dtype]
        opt = Options()
        lib().alto_options_init(ctypes.byref(opt))
        opt.key_bits = key_bits
        opt.nparts = nparts
        opt.use_flags = 1 if use_flags else 0
        if variants is not None:
            for n, v in enumerate(variants):
                opt.variant[n] = int(v)
        self._cbs = None
        if allocator is not None:
            a, f = allocator
            self._cbs = (_ALLOC_FN(a), _FREE_FN(f))
            opt.alloc, opt.free = self._cbs
        ptrs = (ctypes.c_void_p * max(N, 1))(*[a.data_ptr() for a in idx])
        h = ctypes.c_void_p()
        self._h = None
        _check(lib().alto_create(ctypes.byref(h), N, _dims(self.dims), M, ptrs, idx_bytes,
                                 ctypes.c_void_p(vals.data_ptr()), self.vdtype, ctypes.byref(opt),
                                 _stream(stream)))
        self._h = h
        self.nnz = M

    # -- queries ------------------------------------------------------------
    def layout(self):
        N = self.N
        nm = ctypes.c_int()
        bits = (ctypes.c_int * N)()
        masks = (ctypes.c_uint64 * (2 * N))()
        kw = ctypes.c_int()
        fb = (ctypes.c_int * N)()
        hb = (ctypes.c_int * N)()
        _check(lib().alto_get_layout(self._h, ctypes.byref(nm), bits, masks, ctypes.byref(kw), fb, hb))
        return dict(bits=list(bits), masks=[(masks[2 * n], masks[2 * n + 1]) for n in range(N)],
                    key_words=kw.value, flag_bit=list(fb), hot_bit=list(hb))

    def hot_rows(self, mode):
        """The mode's hot rows, hottest first (uint32 numpy array)."""
        import numpy as np
        rows = np.zeros(1024, dtype=np.uint32)
        n = ctypes.c_int()
        _check(lib().alto_get_hot_rows(self._h, mode, rows.ctypes.data_as(ctypes.c_void_p), ctypes.byref(n)))
        return rows[:n.value].copy()

    def stats(self):
        N = self.N
        nnz = ctypes.c_int64()
        L = ctypes.c_int64()
        d = (ctypes.c_uint64 * N)()
        r = (ctypes.c_double * N)()
        v = (ctypes.c_int * N)()
        mi = (ctypes.c_uint64 * N)()
        _check(lib().alto_get_stats(self._h, ctypes.byref(nnz), ctypes.byref(L), d, r, v, mi))
        return dict(nnz=nnz.value, nparts=L.value, distinct=list(d), reuse=list(r), variant=list(v),
                    max_interval=list(mi))

    def export(self):
        """Host copies: keys (M x key_words uint64), perm (uint32), vals,
        bounds (L+1 int64), intervals (L x N x 2 uint32)."""
        import numpy as np
        lay = self.layout()
        st = self.stats()
        M, L = st["nnz"], st["nparts"]
        keys = np.zeros((M, lay["key_words"]), dtype=np.uint64)
        perm = np.zeros(M, dtype=np.uint32)
        vals = np.zeros(M, dtype={F64: np.float64, F32: np.float32, BF16: np.uint16}[self.vdtype])
        bounds = np.zeros(L + 1, dtype=np.int64)
        ivl = np.zeros((L, self.N, 2), dtype=np.uint32)
        vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
        _check(lib().alto_export(self._h, vp(keys), vp(perm), vp(vals), vp(bounds), vp(ivl)))
        if self.vdtype == BF16:  # BF16 bits -> the exact FP32 values
            vals = (vals.astype(np.uint32) << 16).view(np.float32)
        return dict(keys=keys, perm=perm, vals=vals, bounds=bounds, intervals=ivl)

    def mode_stats(self, mode):
        """[I_n, distinct, reuse, max interval, hot rows, hot share, median and
        90th-percentile unit interval width]."""
        out = (ctypes.c_double * 8)()
        _check(lib().alto_get_mode_stats(self._h, mode, out, 8))
        return list(out)

    def unit_fit(self, mode, rows):
        f = ctypes.c_double()
        _check(lib().alto_get_unit_fit(self._h, mode, int(rows), ctypes.byref(f)))
        return f.value

    def set_variant(self, mode, variant):
        _check(lib().alto_set_variant(self._h, mode, int(variant)))

    def set_gram_engine(self, engine):
        """Engine of the CP-ALS Gram matrices (GRAM_AUTO, GRAM_CUDA_CORES,
        GRAM_TENSOR_CORES)."""
        _check(lib().alto_set_gram_engine(self._h, int(engine)))

    def key_bytes(self):
        """Bytes of one stored key in the streamed MTTKRP format."""
        b = ctypes.c_int()
        _check(lib().alto_get_key_bytes(self._h, ctypes.byref(b)))
        return b.value

    def set_parts(self, mode, nparts):
        """Segment count of this mode's ATOMIC / WARPAGG MTTKRPs (0: the
        tensor's own L)."""
        _check(lib().alto_set_parts(self._h, mode, int(nparts)))

    def resolve_variant(self, mode, rank, fdtype=F32, variant=0):
        """The variant an MTTKRP of this mode and rank runs for ``variant``."""
        v = ctypes.c_int()
        _check(lib().alto_resolve_variant(self._h, mode, int(rank), int(fdtype), int(variant), ctypes.byref(v)))
        return v.value

    def check(self, stream=None):
        _check(lib().alto_check(self._h, _stream(stream)))

    # -- compute ------------------------------------------------------------
    def mttkrp(self, mode, factors, out=None, stream=None):
        """Mode-``mode`` MTTKRP; factors: list of N device tensors (I_m x R),
        factors[mode] may be None.  Returns the I_mode x R output."""
        ref = next(f for m, f in enumerate(factors) if m != mode and f is not None) \
            if self.N > 1 else factors[mode]
        R = int(ref.shape[1])
        fd = _fdtype(ref)
        for m, f in enumerate(factors):
            if m == mode or f is None:
                continue
            if f.dtype != ref.dtype or not f.is_cuda or not f.is_contiguous() or f.shape != (self.dims[m], R):
                raise ValueError("factor %d must be a contiguous CUDA %s tensor of shape (%d, %d)"
                                 % (m, ref.dtype, self.dims[m], R))
        odt = torch.float64 if fd == F64 else torch.float32
        if out is None:
            out = torch.empty((self.dims[mode], R), dtype=odt, device=ref.device)
        elif out.dtype != odt or out.shape != (self.dims[mode], R) or not out.is_contiguous():
            raise ValueError("out must be a contiguous %s tensor of shape (%d, %d)" % (odt, self.dims[mode], R))
        ptrs = (ctypes.c_void_p * self.N)(*[(f.data_ptr() if f is not None else 0) for f in factors])
        _check(lib().alto_mttkrp(self._h, mode, ptrs, R, fd, ctypes.c_void_p(out.data_ptr()), _stream(stream)))
        return out

    def transpose(self, modes, order=False, src=True, idx=True, vals=True, idx_dtype=torch.int64,
                  device=None, stream=None):
        """Sparse tensor transposition (Sec. 5): the nonzeros in the
        lexicographic order of the coordinates of ``modes`` (first mode most
        significant), by a radix sort over those modes' key bits only; ties
        keep ALTO order.  Returns a dict of device tensors: ``order`` (ALTO
        positions) and ``src`` (input positions) as int32 holding uint32
        values, ``idx`` (N coordinate arrays, output mode j = modes[j], the
        other modes after in ascending order) and ``vals`` (stored dtype)."""
        modes = [int(m) for m in modes]
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        M = self.nnz
        res = {}
        if order:
            res["order"] = torch.empty(M, dtype=torch.int32, device=dev)
        if src:
            res["src"] = torch.empty(M, dtype=torch.int32, device=dev)
        if idx:
            if idx_dtype not in (torch.int64, torch.int32):
                raise ValueError("idx_dtype must be int64 or int32")
            res["idx"] = [torch.empty(M, dtype=idx_dtype, device=dev) for _ in range(self.N)]
        if vals:
            vdt = {F64: torch.float64, F32: torch.float32, BF16: torch.bfloat16}[self.vdtype]
            res["vals"] = torch.empty(M, dtype=vdt, device=dev)
        sel = (ctypes.c_int * max(len(modes), 1))(*modes)
        ptr = lambda k: ctypes.c_void_p(res[k].data_ptr()) if k in res else None  # noqa: E731
        iptrs = (ctypes.c_void_p * self.N)(*[a.data_ptr() for a in res["idx"]]) if idx else None
        _check(lib().alto_transpose(self._h, len(modes), sel, ptr("order"), ptr("src"), iptrs,
                                    8 if idx_dtype == torch.int64 else 4, ptr("vals"), _stream(stream)))
        return res

    def cpals(self, factors, iters, lam=None, stream=None, fit=True):
        """Run CP-ALS in place on ``factors``; returns (lambda, fits)."""
        R = int(factors[0].shape[1])
        fd = _fdtype(factors[0])
        for m, f in enumerate(factors):
            if f.dtype != factors[0].dtype or not f.is_cuda or not f.is_contiguous() or f.shape != (self.dims[m], R):
                raise ValueError("factor %d has the wrong dtype, device or shape" % m)
        if lam is None:
            lam = torch.empty(R, dtype=torch.float64, device=factors[0].device)
        ptrs = (ctypes.c_void_p * self.N)(*[f.data_ptr() for f in factors])
        fits = (ctypes.c_double * max(iters, 1))()
        _check(lib().alto_cpals(self._h, R, iters, ptrs, fd, ctypes.c_void_p(lam.data_ptr()),
                                fits if fit else None, _stream(stream)))
        return lam, (list(fits)[:iters] if fit else None)

    def profile(self, enable=True):
        """Time every MTTKRP call of this tensor with CUDA events."""
        _check(lib().alto_profile(self._h, 1 if enable else 0))

    def profile_read(self):
        """(ms per mode, calls per mode) since the previous read."""
        ms = (ctypes.c_double * self.N)()
        calls = (ctypes.c_int64 * self.N)()
        _check(lib().alto_profile_read(self._h, ms, calls))
        return list(ms), list(calls)

    def close(self):
        if getattr(self, "_h", None):
            lib().alto_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

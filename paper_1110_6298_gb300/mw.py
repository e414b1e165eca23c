"""Thin ctypes binding of libmw (include/mw.h).

Argument marshalling only: every step of every transform runs in the CUDA
library.  If libmw.so is missing or cannot be loaded this module raises; there
is no CPU fallback.  Tensors are complex128, on a CUDA device (the call is
enqueued on torch's current stream of that device) or in host memory (the
library stages them through its own device buffers).
"""
import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmw.so")

MW_OK, MW_EINVAL, MW_ENOMEM, MW_ECUDA, MW_ETIMEOUT, MW_EUNSUPPORTED = range(6)
PRECISIONS = {"fp64": 0, "mixed": 1, "mixed_bf16": 1, "mixed_tf32": 2}
FLAG_GRAPH = 1 << 8
FLAG_REAL = 1 << 9
FLAG_DELTA_TN = 1 << 10
FLAG_DELTA_RISBO = 1 << 11
FLAG_AUTOTUNE = 1 << 12
# Wigner-plane recursion: None = the library's default (Trapani-Navaza on the
# mixed precisions, Risbo on FP64); "tn" (mixed only) or "risbo" to choose
DELTA = {None: 0, "tn": FLAG_DELTA_TN, "risbo": FLAG_DELTA_RISBO}

_lib = None


class Tuning(ctypes.Structure):
    """mw_tuning: planes per recursion + contraction launch, spin groups per
    contraction pass, Trapani-Navaza columns per block, measured ms."""
    _fields_ = [("chunk", ctypes.c_int), ("groups", ctypes.c_int), ("tn_threads", ctypes.c_int),
                ("ms", ctypes.c_double)]

    def as_dict(self):
        return {"chunk": self.chunk, "groups": self.groups, "tn_threads": self.tn_threads, "ms": self.ms}


class MWError(RuntimeError):
    def __init__(self, status, what):
        self.status = status
        super().__init__(f"{what}: {status_string(status)}")


def lib():
    """Load libmw.so (raises OSError/RuntimeError if it is absent)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libmw.so not built ({LIB_PATH}); run paper_1110_6298_gb300/build.py")
        L = ctypes.CDLL(LIB_PATH)
        vp, c_int, c_uint, c_size = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint, ctypes.c_size_t
        L.mw_plan_create.argtypes = [ctypes.POINTER(vp), c_int, c_int, c_int, c_uint]
        L.mw_plan_create_spins.argtypes = [ctypes.POINTER(vp), c_int, c_int, ctypes.POINTER(c_int), c_uint]
        L.mw_plan_create_ragged.argtypes = [ctypes.POINTER(vp), c_int, ctypes.POINTER(c_int), ctypes.POINTER(c_int),
                                            c_uint]
        L.mw_plan_create_ragged.restype = c_int
        L.mw_plan_map_elems.argtypes = [vp]
        L.mw_plan_map_elems.restype = c_size
        L.mw_plan_flm_elems.argtypes = [vp]
        L.mw_plan_flm_elems.restype = c_size
        for name in ("mw_forward", "mw_inverse", "mw_forward_adjoint", "mw_inverse_adjoint"):
            getattr(L, name).argtypes = [vp, vp, vp, vp]
            getattr(L, name).restype = c_int
        L.mw_plan_create.restype = c_int
        L.mw_plan_create_spins.restype = c_int
        L.mw_plan_destroy.argtypes = [vp]
        L.mw_plan_destroy.restype = c_int
        L.mw_status_string.argtypes = [c_int]
        L.mw_status_string.restype = ctypes.c_char_p
        L.mw_map_size.argtypes = [c_int]
        L.mw_map_size.restype = c_size
        L.mw_flm_size.argtypes = [c_int]
        L.mw_flm_size.restype = c_size
        L.mw_plan_workspace_bytes.argtypes = [vp]
        L.mw_plan_workspace_bytes.restype = c_size
        L.mw_plan_last_launches.argtypes = [vp]
        L.mw_plan_last_launches.restype = c_int
        L.mw_plan_fft_bluestein.argtypes = [vp]
        L.mw_plan_fft_bluestein.restype = c_int
        L.mw_plan_sync.argtypes = [vp, vp]
        L.mw_plan_sync.restype = c_int
        L.mw_plan_set_timing.argtypes = [vp, c_int]
        L.mw_plan_set_timing.restype = c_int
        L.mw_plan_stage_times.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong),
                                          c_int]
        L.mw_plan_stage_times.restype = c_int
        L.mw_quadrature_weights.argtypes = [c_int, c_int, vp, vp]
        L.mw_quadrature_weights.restype = c_int
        L.mw_quadrature.argtypes = [vp, vp, vp, vp]
        L.mw_quadrature.restype = c_int
        L.mw_forward_inverse.argtypes = [vp, vp, vp, vp, vp, vp]
        L.mw_forward_inverse.restype = c_int
        L.mw_inverse_noalloc.argtypes = [c_int, c_int, vp, vp, vp]
        L.mw_inverse_noalloc.restype = c_int
        ll = ctypes.c_longlong
        L.mw_plan_batch.argtypes = [vp]
        L.mw_plan_batch.restype = c_int
        for name in ("mw_plan_band_limit", "mw_plan_spin"):
            getattr(L, name).argtypes = [vp, c_int]
            getattr(L, name).restype = c_int
        for name in ("mw_plan_map_offset", "mw_plan_flm_offset"):
            getattr(L, name).argtypes = [vp, c_int]
            getattr(L, name).restype = ll
        L.mw_layout_ragged.argtypes = [c_int, ctypes.POINTER(c_int), ctypes.POINTER(ll), ctypes.POINTER(ll)]
        L.mw_layout_ragged.restype = c_int
        L.mw_plan_get_tuning.argtypes = [vp, ctypes.POINTER(Tuning)]
        L.mw_plan_get_tuning.restype = c_int
        L.mw_plan_set_tuning.argtypes = [vp, ctypes.POINTER(Tuning)]
        L.mw_plan_set_tuning.restype = c_int
        L.mw_plan_autotune.argtypes = [vp, vp]
        L.mw_plan_autotune.restype = c_int
        L.mw_tune_key.argtypes = [c_int, ctypes.POINTER(c_int), ctypes.POINTER(c_int), c_uint, ctypes.c_char_p,
                                  ctypes.c_char_p, c_size]
        L.mw_tune_key.restype = c_int
        L.mw_tune_cache_lookup.argtypes = [ctypes.c_char_p, ctypes.c_char_p, ctypes.POINTER(Tuning),
                                           ctypes.POINTER(c_int)]
        L.mw_tune_cache_lookup.restype = c_int
        L.mw_tune_cache_store.argtypes = [ctypes.c_char_p, ctypes.c_char_p, ctypes.POINTER(Tuning)]
        L.mw_tune_cache_store.restype = c_int
        _lib = L
    return _lib


def status_string(st):
    return lib().mw_status_string(int(st)).decode()


def map_size(L):
    return int(lib().mw_map_size(int(L)))


def flm_size(L):
    return int(lib().mw_flm_size(int(L)))


def layout_ragged(Ls):
    """(map_offsets, flm_offsets), each of len(Ls) + 1 entries (the last is
    the total), as the library lays out a ragged batch of band limits Ls."""
    n = len(Ls)
    la = (ctypes.c_int * n)(*[int(x) for x in Ls])
    mo = (ctypes.c_longlong * (n + 1))()
    fo = (ctypes.c_longlong * (n + 1))()
    st = lib().mw_layout_ragged(n, la, mo, fo)
    if st != MW_OK:
        raise MWError(st, "mw_layout_ragged")
    return list(mo), list(fo)


def tune_key(Ls, spins, flags, device):
    """The tuning-cache key of a plan of maps (Ls[b], spins[b]) with `flags` on
    the named device (host-only)."""
    n = len(Ls)
    buf = ctypes.create_string_buffer(64 + 24 * n + 256)
    st = lib().mw_tune_key(n, (ctypes.c_int * n)(*Ls), (ctypes.c_int * n)(*spins), int(flags),
                           device.encode(), buf, len(buf))
    if st != MW_OK:
        raise MWError(st, "mw_tune_key")
    return buf.value.decode()


def tune_cache_lookup(path, key):
    """The tuning stored under `key` in the cache file, or None."""
    t, found = Tuning(), ctypes.c_int(0)
    st = lib().mw_tune_cache_lookup(str(path).encode(), key.encode(), ctypes.byref(t), ctypes.byref(found))
    if st != MW_OK:
        raise MWError(st, "mw_tune_cache_lookup")
    return t.as_dict() if found.value else None


def tune_cache_store(path, key, chunk, groups, tn_threads, ms=0.0):
    st = lib().mw_tune_cache_store(str(path).encode(), key.encode(),
                                   ctypes.byref(Tuning(int(chunk), int(groups), int(tn_threads), float(ms))))
    if st != MW_OK:
        raise MWError(st, "mw_tune_cache_store")


def quadrature_size(L):
    """Samples of a map in the quadrature layout: L(L-1) + 1."""
    return int(L) * (int(L) - 1) + 1


def quadrature_weights(L, s=0, device="cuda"):
    """q(theta_t), t = 0..L-1, of the MW quadrature rule (Sec. IV-F), computed on the GPU."""
    q = torch.empty(int(L), dtype=torch.float64, device=device)
    st = lib().mw_quadrature_weights(int(L), int(s), ctypes.c_void_p(q.data_ptr()), _stream_of(q))
    if st != MW_OK:
        raise MWError(st, "mw_quadrature_weights")
    return q


def _stream_of(t):
    if t.is_cuda:
        return ctypes.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class Plan:
    """A transform plan: L, one spin per map (or one spin for all), precision."""

    def __init__(self, L, spins, batch=None, precision="fp64", graph=False, delta=None, autotune=False):
        if isinstance(spins, int):
            if batch is None:
                batch = 1
            spins = [spins] * int(batch)
        spins = [int(s) for s in spins]
        if batch is not None and int(batch) != len(spins):
            raise ValueError("batch does not match len(spins)")
        self.L, self.spins, self.batch = int(L), spins, len(spins)
        self.precision = precision
        h = ctypes.c_void_p()
        arr = (ctypes.c_int * len(spins))(*spins)
        flags = PRECISIONS[precision] | (FLAG_GRAPH if graph else 0) | DELTA[delta] | (FLAG_AUTOTUNE if autotune else 0)
        st = lib().mw_plan_create_spins(ctypes.byref(h), self.L, self.batch, arr, flags)
        if st != MW_OK:
            raise MWError(st, "mw_plan_create_spins")
        self._h = h
        self._nmap = self.batch * map_size(self.L)
        self._nflm = self.batch * flm_size(self.L)

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().mw_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def layout(self):
        """[(L, spin, map_offset, flm_offset)] per map, as the plan lays out
        its buffers (read from the library)."""
        h = self._h
        n = int(lib().mw_plan_batch(h))
        return [(int(lib().mw_plan_band_limit(h, b)), int(lib().mw_plan_spin(h, b)),
                 int(lib().mw_plan_map_offset(h, b)), int(lib().mw_plan_flm_offset(h, b))) for b in range(n)]

    @property
    def tuning(self):
        """The plan's tuning as a dict (chunk, groups, tn_threads, ms)."""
        t = Tuning()
        st = lib().mw_plan_get_tuning(self._h, ctypes.byref(t))
        if st != MW_OK:
            raise MWError(st, "mw_plan_get_tuning")
        return t.as_dict()

    def set_tuning(self, chunk, groups, tn_threads, ms=0.0):
        t = Tuning(int(chunk), int(groups), int(tn_threads), float(ms))
        st = lib().mw_plan_set_tuning(self._h, ctypes.byref(t))
        if st != MW_OK:
            raise MWError(st, "mw_plan_set_tuning")

    def autotune(self, stream=None):
        """Time the tuning candidates on this plan's shapes and keep the fastest."""
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        st = lib().mw_plan_autotune(self._h, ctypes.c_void_p(stream))
        if st != MW_OK:
            raise MWError(st, "mw_plan_autotune")
        return self.tuning

    @property
    def workspace_bytes(self):
        return int(lib().mw_plan_workspace_bytes(self._h))

    @property
    def last_launches(self):
        return int(lib().mw_plan_last_launches(self._h))

    @property
    def fft_bluestein(self):
        """True if the length-(2L-1) DFTs run by Bluestein's convolution."""
        return bool(lib().mw_plan_fft_bluestein(self._h) == 1)

    def sync(self, stream=None):
        """Wait for this plan's work and raise MWError on a device-side timeout."""
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        st = lib().mw_plan_sync(self._h, ctypes.c_void_p(stream))
        if st != MW_OK:
            raise MWError(st, "mw_plan_sync")

    STAGES = ("phi", "theta", "delta", "contract")

    def set_timing(self, enable=True):
        st = lib().mw_plan_set_timing(self._h, int(bool(enable)))
        if st != MW_OK:
            raise MWError(st, "mw_plan_set_timing")

    def stage_times(self, reset=False):
        """{stage: (milliseconds, launches)} accumulated since the last reset."""
        ms = (ctypes.c_double * 4)()
        nl = (ctypes.c_longlong * 4)()
        st = lib().mw_plan_stage_times(self._h, ms, nl, int(bool(reset)))
        if st != MW_OK:
            raise MWError(st, "mw_plan_stage_times")
        return {k: (ms[i], nl[i]) for i, k in enumerate(self.STAGES)}

    def _call(self, name, x, n_in, n_out, out):
        if x.dtype != torch.complex128:
            raise TypeError("expected a complex128 tensor")
        if x.numel() != n_in:
            raise ValueError(f"expected {n_in} elements, got {tuple(x.shape)}")
        x = x.contiguous()
        if out is None:
            shape = (self.batch, n_out // self.batch) if n_out % self.batch == 0 and self._uniform else (n_out,)
            out = torch.empty(shape, dtype=torch.complex128, device=x.device)
        elif out.dtype != torch.complex128 or out.numel() != n_out or not out.is_contiguous():
            raise ValueError("bad output tensor")
        st = getattr(lib(), name)(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                  _stream_of(x))
        if st != MW_OK:
            raise MWError(st, name)
        return out

    _uniform = True

    def forward(self, maps, out=None):
        return self._call("mw_forward", maps, self._nmap, self._nflm, out)

    def inverse(self, flm, out=None):
        return self._call("mw_inverse", flm, self._nflm, self._nmap, out)

    def forward_inverse(self, maps, flm, flm_out=None, map_out=None):
        """Forward of `maps` and inverse of `flm` (independent inputs) sharing one
        Wigner-Delta recursion; returns (flm_out, map_out)."""
        for x, n in ((maps, self._nmap), (flm, self._nflm)):
            if x.dtype != torch.complex128:
                raise TypeError("expected complex128 tensors")
            if x.numel() != n:
                raise ValueError(f"expected {n} elements, got {tuple(x.shape)}")
        maps, flm = maps.contiguous(), flm.contiguous()

        def make(o, n, like):
            if o is None:
                shape = (self.batch, n // self.batch) if self._uniform else (n,)
                return torch.empty(shape, dtype=torch.complex128, device=like.device)
            if o.dtype != torch.complex128 or o.numel() != n or not o.is_contiguous():
                raise ValueError("bad output tensor")
            return o

        flm_out = make(flm_out, self._nflm, maps)
        map_out = make(map_out, self._nmap, flm)
        st = lib().mw_forward_inverse(self._h, ctypes.c_void_p(maps.data_ptr()), ctypes.c_void_p(flm_out.data_ptr()),
                                      ctypes.c_void_p(flm.data_ptr()), ctypes.c_void_p(map_out.data_ptr()),
                                      _stream_of(maps))
        if st != MW_OK:
            raise MWError(st, "mw_forward_inverse")
        return flm_out, map_out

    def quadrature(self, maps_q, out=None):
        """Integrals over the sphere (Sec. IV-F) of the batch of maps in the
        quadrature layout [batch][L(L-1)+1] (CUDA complex128); returns [batch]."""
        n = self.batch * quadrature_size(self.L)
        if maps_q.dtype != torch.complex128 or not maps_q.is_cuda or maps_q.numel() != n:
            raise ValueError(f"expected a complex128 CUDA tensor of {n} elements")
        maps_q = maps_q.contiguous()
        if out is None:
            out = torch.empty(self.batch, dtype=torch.complex128, device=maps_q.device)
        st = lib().mw_quadrature(self._h, ctypes.c_void_p(maps_q.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                 _stream_of(maps_q))
        if st != MW_OK:
            raise MWError(st, "mw_quadrature")
        return out

    def forward_adjoint(self, flm, out=None):
        return self._call("mw_forward_adjoint", flm, self._nflm, self._nmap, out)

    def inverse_adjoint(self, maps, out=None):
        return self._call("mw_inverse_adjoint", maps, self._nmap, self._nflm, out)


class RealPlan(Plan):
    """`batch` real scalar maps (Sec. IV-G): maps are float64 [batch][N_MW],
    coefficients complex128 [batch][L*L].

    forward returns coefficients that satisfy f_{l,-m} = (-1)^m conj(f_lm)
    exactly; inverse returns the real part of the synthesis of the given
    coefficients.  The library carries two real maps per complex transform, so
    a batch of B real maps costs a complex batch of ceil(B/2).  No adjoints or
    quadrature on real plans."""

    def __init__(self, L, batch=1, precision="fp64", graph=False, delta=None):
        self.L, self.batch, self.spins = int(L), int(batch), [0] * int(batch)
        self.precision = precision
        h = ctypes.c_void_p()
        flags = PRECISIONS[precision] | FLAG_REAL | (FLAG_GRAPH if graph else 0) | DELTA[delta]
        st = lib().mw_plan_create(ctypes.byref(h), self.L, 0, self.batch, flags)
        if st != MW_OK:
            raise MWError(st, "mw_plan_create (real)")
        self._h = h
        self._nmap = self.batch * map_size(self.L)
        self._nflm = self.batch * flm_size(self.L)

    def _rcall(self, name, x, in_dtype, n_in, out_dtype, n_out, out):
        if x.dtype != in_dtype:
            raise TypeError(f"expected a {in_dtype} tensor")
        if x.numel() != n_in:
            raise ValueError(f"expected {n_in} elements, got {tuple(x.shape)}")
        x = x.contiguous()
        if out is None:
            out = torch.empty((self.batch, n_out // self.batch), dtype=out_dtype, device=x.device)
        elif out.dtype != out_dtype or out.numel() != n_out or not out.is_contiguous():
            raise ValueError("bad output tensor")
        st = getattr(lib(), name)(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                  _stream_of(x))
        if st != MW_OK:
            raise MWError(st, name)
        return out

    def forward(self, maps, out=None):
        return self._rcall("mw_forward", maps, torch.float64, self._nmap, torch.complex128, self._nflm, out)

    def inverse(self, flm, out=None):
        return self._rcall("mw_inverse", flm, torch.complex128, self._nflm, torch.float64, self._nmap, out)

    def forward_inverse(self, maps, flm, flm_out=None, map_out=None):
        """Forward of the real `maps` and inverse of `flm` sharing one
        Wigner-Delta recursion; returns (flm_out, map_out)."""
        for x, dt, n in ((maps, torch.float64, self._nmap), (flm, torch.complex128, self._nflm)):
            if x.dtype != dt:
                raise TypeError(f"expected {dt}")
            if x.numel() != n:
                raise ValueError(f"expected {n} elements, got {tuple(x.shape)}")
        maps, flm = maps.contiguous(), flm.contiguous()

        def make(o, n, dt, like):
            if o is None:
                return torch.empty((self.batch, n // self.batch), dtype=dt, device=like.device)
            if o.dtype != dt or o.numel() != n or not o.is_contiguous():
                raise ValueError("bad output tensor")
            return o

        flm_out = make(flm_out, self._nflm, torch.complex128, maps)
        map_out = make(map_out, self._nmap, torch.float64, flm)
        st = lib().mw_forward_inverse(self._h, ctypes.c_void_p(maps.data_ptr()), ctypes.c_void_p(flm_out.data_ptr()),
                                      ctypes.c_void_p(flm.data_ptr()), ctypes.c_void_p(map_out.data_ptr()),
                                      _stream_of(maps))
        if st != MW_OK:
            raise MWError(st, "mw_forward_inverse")
        return flm_out, map_out

    def forward_adjoint(self, flm, out=None):
        raise MWError(MW_EUNSUPPORTED, "forward_adjoint on a real plan")

    def inverse_adjoint(self, maps, out=None):
        raise MWError(MW_EUNSUPPORTED, "inverse_adjoint on a real plan")

    def quadrature(self, maps_q, out=None):
        raise MWError(MW_EUNSUPPORTED, "quadrature on a real plan")


class RaggedPlan(Plan):
    """n maps of their own band limits Ls[b] and spins spins[b] in one plan.

    Buffers are flat: the maps (resp. f_lm blocks) back to back in the given
    order; map_offsets / flm_offsets give where each starts."""

    _uniform = False

    def __init__(self, Ls, spins, precision="mixed", graph=False, delta=None):
        Ls = [int(x) for x in Ls]
        spins = [int(x) for x in spins]
        if len(Ls) != len(spins):
            raise ValueError("Ls and spins differ in length")
        self.Ls, self.spins, self.batch, self.L = Ls, spins, len(Ls), max(Ls)
        self.precision = precision
        h = ctypes.c_void_p()
        la = (ctypes.c_int * len(Ls))(*Ls)
        sa = (ctypes.c_int * len(spins))(*spins)
        flags = PRECISIONS[precision] | (FLAG_GRAPH if graph else 0) | DELTA[delta]
        st = lib().mw_plan_create_ragged(ctypes.byref(h), len(Ls), la, sa, flags)
        if st != MW_OK:
            raise MWError(st, "mw_plan_create_ragged")
        self._h = h
        self._nmap = int(lib().mw_plan_map_elems(h))
        self._nflm = int(lib().mw_plan_flm_elems(h))
        lay = self.layout()
        self.map_offsets = [x[2] for x in lay]
        self.flm_offsets = [x[3] for x in lay]


NOALLOC_MAX_L = 128


def inverse_noalloc(L, s, flm, out):
    """Inverse transform of one map without any device allocation.

    For callers that cannot allocate device memory (inside a custom
    allocator's callbacks, hosts that forbid allocation after start-up,
    processes whose free device memory belongs to another pool): the library
    keeps every intermediate in one static device array of about 2.6 MB, so
    the caller provides both buffers.  flm: L*L complex128 on the current CUDA
    device; out: N_MW complex128 on that device.  L <= NOALLOC_MAX_L.  Calls
    share the static array, so calls whose GPU work overlaps (two streams or
    threads) race; calls made outside a stream capture look the array's
    address up, so one such call on each device should precede any stream
    capture.  Returns out.
    """
    for name, t, n in (("flm", flm, flm_size(L)), ("out", out, map_size(L))):
        if t.dtype != torch.complex128 or not t.is_cuda or not t.is_contiguous() or t.numel() != n:
            raise ValueError(f"{name}: expected a contiguous complex128 CUDA tensor of {n} elements")
    st = lib().mw_inverse_noalloc(int(L), int(s), ctypes.c_void_p(flm.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                  _stream_of(flm))
    if st != MW_OK:
        raise MWError(st, f"mw_inverse_noalloc(L={L}, s={s}; at most L={NOALLOC_MAX_L})")
    return out

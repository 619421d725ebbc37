"""ctypes binding of libcm.so (the C ABI declared in include/*.h).

Argument marshalling only: every step of the extraction runs in the library's
CUDA kernels.  Tensors are used for device memory and streams; the library
sees raw pointers, sizes and a cudaStream_t.  If the library is missing the
binding raises: there is no fallback path.
"""

from __future__ import annotations

import ctypes
import os
import re

from . import build as _build

TOEPLITZ, CIRCULANT, DODIS = 0, 1, 2

STATUS = {0: "CM_OK", 1: "CM_EINVAL", 2: "CM_EPRECOND", 3: "CM_ENOMEM", 4: "CM_EAGAIN",
          5: "CM_ETIMEDOUT", 6: "CM_EDEVICE", 7: "CM_ENOTFOUND"}
CM_OK, CM_EINVAL, CM_EPRECOND, CM_ENOMEM, CM_EAGAIN, CM_ETIMEDOUT, CM_EDEVICE, CM_ENOTFOUND = range(8)
FLAG_PRECOND, FLAG_TIMEOUT = 0x1, 0x2

_lib = None

_P = ctypes.c_void_p
_U64 = ctypes.c_uint64
_U32 = ctypes.c_uint32
_I = ctypes.c_int

# name -> (restype, argtypes)
PROTOTYPES = {
    "cm_create": (_I, [ctypes.POINTER(_P), _I, _P]),
    "cm_destroy": (None, [_P]),
    "cm_status_str": (ctypes.c_char_p, [_I]),
    "cm_toeplitz": (_I, [_P, _P, _U64, _P, _U64, _P, _P]),
    "cm_circulant": (_I, [_P, _P, _U64, _P, _U64, _P, _P]),
    "cm_dodis": (_I, [_P, _P, _P, _U64, _U64, _P, _P]),
    "cm_compose": (_I, [_P, _I, _P, _U64, _P, _U64, _I, _U64, _U64, _P, _P]),
    "cm_calibrate": (_I, [_P, ctypes.c_char_p, _U32, _U32]),
    "cm_tune_query": (_I, [_P, _U32, _U32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                           ctypes.POINTER(ctypes.c_int32)]),
    "cm_device_status": (_I, [_P, _P, ctypes.POINTER(_U32)]),
    "cm_extract_host": (_I, [_P, _I, _P, _U64, _P, _U64, _P, _P]),
    "cm_toeplitz_noalloc": (_I, [_P, _U64, _P, _U64, _P, _P]),
    "cm_field_selftest": (_I, [_I, _U64, _U64, ctypes.POINTER(_U64)]),
    "cm_batch_toeplitz_shared_seed": (_I, [_P, _P, _U64, _U64, _P, _U64, _P, _I, _P]),
    "cm_shared_seed_engine": (_I, [_U64, _U64]),
    "cm_server_start": (_I, [_P, _P]),
    "cm_server_stop": (_I, [_P]),
    "cm_submit": (_I, [_P, _P, ctypes.POINTER(_U64)]),
    "cm_poll": (_I, [_P, _U64, _P, _U64]),
    "cm_server_get_stats": (_I, [_P, _P]),
    "cm_batch_create": (_I, [_P, _P, _U32, _U32, ctypes.POINTER(_P)]),
    "cm_batch_launch": (_I, [_P, _P]),
    "cm_batch_destroy": (None, [_P]),
    "cm_batch_info": (_I, [_P, _P]),
    "cm_batch_extract": (_I, [_P, _P, _U32, _P]),
    "cm_batch_toeplitz": (_I, [_P, _P, _U32, _P]),
    "cm_profile_enable": (_I, [_P, _I]),
    "cm_profile_read": (_I, [_P, _P, _U32, ctypes.POINTER(_U32), _I]),
    "cm_is_na_prime": (_I, [_U64]),
    "cm_next_na_prime": (_U64, [_U64]),
    "cm_prev_na_prime": (_U64, [_U64]),
    "cm_ntt_length": (_U64, [_I, _U64, _U64]),
    "cm_scratch_bytes": (_U64, [_I, _U64, _U64]),
    "cm_launch_count": (_U32, [_I, _U64, _U64]),
    "cm_block_count": (_U64, [_I, _U64, _U64, _U32]),
    "cm_plan_query": (_I, [_I, _U64, _U64, ctypes.c_void_p, ctypes.c_void_p]),
    "cm_modmul_rate": (_I, [_I, _U32, ctypes.POINTER(ctypes.c_double)]),
    "cm_rsh_field_bits": (_U32, [_U64, ctypes.c_double]),
    "cm_rsh_modulus": (_I, [_U32, ctypes.POINTER(_U32), ctypes.POINTER(_U32)]),
    "cm_trevisan_rsh": (_I, [ctypes.c_void_p, ctypes.c_void_p, _U64, _U32, ctypes.c_void_p, _U64, ctypes.c_void_p,
                             ctypes.c_void_p]),
    "cm_trevisan": (_I, [ctypes.c_void_p, ctypes.c_void_p, _U64, ctypes.c_void_p, _U64, ctypes.c_void_p, _U32,
                         _U64, _U32, ctypes.c_void_p, ctypes.c_void_p]),
    "cm_plan_products": (_I, [_I, _U64, _U64, ctypes.c_void_p, ctypes.c_void_p, _U64, ctypes.POINTER(_U64)]),
    "cm_output_length": (_I, [_I, _I, _I, _U64, _U64, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                              ctypes.POINTER(ctypes.c_int64)]),
    "cm_trevisan_seed_length": (_I, [_U64, _U64, ctypes.c_double, ctypes.POINTER(_U64),
                                     ctypes.POINTER(_U64), ctypes.POINTER(_U64)]),
    "cm_plan_params": (_I, [_I, _I, _I, _U64, ctypes.c_double, ctypes.c_double, ctypes.c_double, _I, _P]),
    "cm_closest_na_prime": (_U64, [_U64]),
    "cm_von_neumann": (_I, [_P, _P, _U64, _P, _P, _P]),
    "cm_von_neumann_host": (_I, [_P, _P, _U64, _P, ctypes.POINTER(_U64), _P]),
    "cm_von_neumann_scratch_bytes": (_U64, [_U64]),
}

TREVISAN = 3
MODEL_SEEDED, MODEL_PRODUCT, MODEL_MARKOV = 0, 1, 2
ADV_CLASSICAL, ADV_QUANTUM = 0, 1
ADJUST_UP, ADJUST_DOWN, ADJUST_CLOSEST = 0, 1, 2
FIELD_AUTO, FIELD_GOLDILOCKS, FIELD_Q30, FIELD_Q25 = 0, 1, 2, 3
TUNE_FORCE = 1
SERVER_NO_EXPRESS = 0xFFFFFFFF
PLAN_COST, PLAN_SINGLE = 0, 1


class Options(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_uint64), ("max_transform_lg", ctypes.c_uint32),
                ("field", ctypes.c_uint32), ("max_sum_blocks", ctypes.c_uint32),
                ("plan_mode", ctypes.c_uint32), ("reserved", ctypes.c_uint32 * 4)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("transform_length", ctypes.c_uint64), ("products", ctypes.c_uint64),
                ("windows", ctypes.c_uint64), ("scratch_bytes", ctypes.c_uint64),
                ("launches", ctypes.c_uint32), ("field", ctypes.c_uint32), ("est_ms", ctypes.c_double),
                ("tail_terms", ctypes.c_uint64), ("reserved", ctypes.c_uint64 * 3)]


class ProductDesc(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in ("K", "m", "L", "zword", "a_len", "a_srclen", "a_off",
                                               "b_len", "b_srclen", "b_off")] + \
               [("a_mode", ctypes.c_uint32), ("b_mode", ctypes.c_uint32), ("field", ctypes.c_uint32),
                ("sum", ctypes.c_int32), ("xor_into", ctypes.c_uint32), ("tail_terms", ctypes.c_uint32)]


class ParamPlan(ctypes.Structure):
    _fields_ = [("n1", ctypes.c_uint64), ("n2", ctypes.c_uint64), ("pad_input", ctypes.c_uint64),
                ("cut_input", ctypes.c_uint64), ("k1", ctypes.c_double), ("k2", ctypes.c_double),
                ("m", ctypes.c_int64), ("reserved", ctypes.c_uint64 * 3)]


class ProfileEntry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 40), ("launches", ctypes.c_uint64),
                ("total_ms", ctypes.c_double)]


class CmDesc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("reserved", ctypes.c_uint32), ("n", ctypes.c_uint64),
                ("m", ctypes.c_uint64), ("x", ctypes.c_void_p), ("y", ctypes.c_void_p),
                ("z", ctypes.c_void_p)]


class BatchStats(ctypes.Structure):
    _fields_ = [("instances", ctypes.c_uint32), ("work_items", ctypes.c_uint32),
                ("solo_instances", ctypes.c_uint32), ("tile_lg", ctypes.c_uint32),
                ("grid", ctypes.c_uint32), ("graph", ctypes.c_uint32),
                ("scratch_bytes", ctypes.c_uint64), ("kernel_launches", ctypes.c_uint64),
                ("output_bits", ctypes.c_uint64), ("transform_elements", ctypes.c_uint64)]


class CmRequest(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("flags", ctypes.c_uint32), ("n", ctypes.c_uint64),
                ("m", ctypes.c_uint64), ("x", ctypes.c_void_p), ("y", ctypes.c_void_p),
                ("z", ctypes.c_void_p), ("seed_id", ctypes.c_uint64), ("user", ctypes.c_uint64)]


REQ_SEED_CACHE = 0x1


class CmResult(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("reserved", ctypes.c_uint32), ("t_submit_ns", ctypes.c_uint64),
                ("t_admit_ns", ctypes.c_uint64), ("t_done_ns", ctypes.c_uint64), ("wave", ctypes.c_uint64)]


class ServerOptions(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_uint64), ("slots", ctypes.c_uint32),
                ("max_queue", ctypes.c_uint32), ("max_wave", ctypes.c_uint32), ("express_slots", ctypes.c_uint32),
                ("seed_cache_bytes", ctypes.c_uint64), ("reserved", ctypes.c_uint32 * 2)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("rejected", ctypes.c_uint64),
                ("waves", ctypes.c_uint64), ("inflight_bytes", ctypes.c_uint64),
                ("max_inflight_bytes", ctypes.c_uint64), ("budget_bytes", ctypes.c_uint64),
                ("seed_cache_hits", ctypes.c_uint64), ("seed_cache_misses", ctypes.c_uint64),
                ("seed_cache_bytes", ctypes.c_uint64), ("seed_cache_entries", ctypes.c_uint64),
                ("queued", ctypes.c_uint32), ("busy_slots", ctypes.c_uint32), ("slots", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]


BATCH_AUTOTUNE, BATCH_NO_GRAPH, BATCH_TEST_STALL = 0x1, 0x2, 0x4
ENGINE_AUTO, ENGINE_IMMA, ENGINE_GF2, ENGINE_BMMA = 0, 1, 2, 3


class CMError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {STATUS.get(status, status)}" if what else STATUS.get(status, str(status)))


def header_functions() -> list[str]:
    """Names of the functions the headers under include/ declare."""
    names = set()
    for h in sorted(os.listdir(_build.INCLUDE)):
        if not h.endswith(".h"):
            continue
        with open(os.path.join(_build.INCLUDE, h)) as f:
            text = re.sub(r"/\*.*?\*/", "", f.read(), flags=re.S)
        names |= set(re.findall(r"\b(cm_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def lib():
    """Load libcm.so (built by build.build()); raise if it is absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(_build.LIB):
            raise RuntimeError(
                "libcm.so is not built; run paper_2402_09481_gb300.build.build() "
                "(there is no CPU fallback)")
        L = ctypes.CDLL(_build.LIB)
        for name, (res, args) in PROTOTYPES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status: int, what: str):
    if status != CM_OK:
        raise CMError(status, what)


def words(nbits: int) -> int:
    return (int(nbits) + 63) // 64


def ntt_length(kind: int, n: int, m: int) -> int:
    return int(lib().cm_ntt_length(kind, n, m))


def scratch_bytes(kind: int, n: int, m: int) -> int:
    return int(lib().cm_scratch_bytes(kind, n, m))


def block_count(kind: int, n: int, m: int, max_transform_lg: int = 0) -> int:
    return int(lib().cm_block_count(kind, n, m, max_transform_lg))


def plan_query(kind: int, n: int, m: int, max_transform_lg: int = 0, field: int = FIELD_AUTO,
               hbm_budget_bytes: int = 0, max_sum_blocks: int = 0, plan_mode: int = PLAN_COST) -> dict:
    """How one call of (kind, n, m) runs under these options (cm_plan_query)."""
    o = Options(hbm_budget_bytes, max_transform_lg, field, max_sum_blocks, plan_mode)
    info = PlanInfo()
    _check(lib().cm_plan_query(kind, n, m, ctypes.byref(o), ctypes.byref(info)), "cm_plan_query")
    return {k: getattr(info, k) for k in ("transform_length", "products", "windows", "scratch_bytes",
                                          "launches", "field", "est_ms", "tail_terms")}


def plan_products(kind: int, n: int, m: int, max_transform_lg: int = 0, field: int = FIELD_AUTO,
                  hbm_budget_bytes: int = 0, max_sum_blocks: int = 0, plan_mode: int = PLAN_COST) -> list[dict]:
    """The middle products of one call's plan (cm_plan_products), in run order."""
    o = Options(hbm_budget_bytes, max_transform_lg, field, max_sum_blocks, plan_mode)
    cnt = ctypes.c_uint64()
    _check(lib().cm_plan_products(kind, n, m, ctypes.byref(o), None, 0, ctypes.byref(cnt)), "cm_plan_products")
    arr = (ProductDesc * max(cnt.value, 1))()
    _check(lib().cm_plan_products(kind, n, m, ctypes.byref(o), arr, cnt.value, ctypes.byref(cnt)),
           "cm_plan_products")
    return [{k: getattr(arr[i], k) for k, _ in ProductDesc._fields_} for i in range(cnt.value)]


def launch_count(kind: int, n: int, m: int) -> int:
    return int(lib().cm_launch_count(kind, n, m))


def rsh_field_bits(n: int, eps1: float) -> int:
    """l = ceil(log2 n + 2 log2(2 / eps1)) of the RSH one-bit extractor."""
    return int(lib().cm_rsh_field_bits(n, eps1))


def rsh_modulus(l: int) -> list[int]:
    """Middle exponents of the GF(2^l) modulus: [k] (trinomial) or [a, b, c]."""
    taps = (_U32 * 3)()
    cnt = _U32()
    _check(lib().cm_rsh_modulus(l, taps, ctypes.byref(cnt)), "cm_rsh_modulus")
    return [int(taps[i]) for i in range(cnt.value)]


def modmul_rate(device: int = 0, field: int = FIELD_Q30) -> float:
    """Measured modular products per second of the field's multiply (cm_modmul_rate)."""
    r = ctypes.c_double()
    _check(lib().cm_modmul_rate(device, field, ctypes.byref(r)), "cm_modmul_rate")
    return r.value


def field_selftest(device: int = 0, count: int = 1 << 20, seed: int = 1) -> int:
    """Number of disagreements between the device field arithmetic and its C form."""
    bad = ctypes.c_uint64(0)
    _check(lib().cm_field_selftest(device, count, seed, ctypes.byref(bad)), "cm_field_selftest")
    return int(bad.value)


def is_na_prime(P: int) -> bool:
    return bool(lib().cm_is_na_prime(P))


def next_na_prime(n: int) -> int:
    return int(lib().cm_next_na_prime(n))


def prev_na_prime(n: int) -> int:
    return int(lib().cm_prev_na_prime(n))


def von_neumann_scratch_bytes(n: int) -> int:
    return int(lib().cm_von_neumann_scratch_bytes(n))


def closest_na_prime(n: int) -> int:
    return int(lib().cm_closest_na_prime(n))


def output_length(kind: int, model: int, adversary: int, n1: int, k1: float, log2_eps: float,
                  k2: float = 0.0, d: int = 0) -> int:
    """Largest m the paper's bound allows (cm_output_length)."""
    m = ctypes.c_int64(0)
    _check(lib().cm_output_length(kind, model, adversary, n1, d, float(k1), float(k2), float(log2_eps),
                                  ctypes.byref(m)), "cm_output_length")
    return int(m.value)


def trevisan_seed_length(n1: int, m: int, log2_eps: float) -> tuple[int, int, int]:
    t, a, d = _U64(0), _U64(0), _U64(0)
    _check(lib().cm_trevisan_seed_length(n1, m, float(log2_eps), ctypes.byref(t), ctypes.byref(a),
                                         ctypes.byref(d)), "cm_trevisan_seed_length")
    return int(t.value), int(a.value), int(d.value)


def plan_params(kind: int, model: int, adversary: int, n_raw: int, k1: float, log2_eps: float,
                seed_rate: float = 1.0, adjust: int = ADJUST_UP) -> dict:
    """Lengths for one extraction (cm_plan_params) as a dict."""
    p = ParamPlan()
    _check(lib().cm_plan_params(kind, model, adversary, n_raw, float(k1), float(seed_rate), float(log2_eps),
                                adjust, ctypes.byref(p)), "cm_plan_params")
    return dict(n1=int(p.n1), n2=int(p.n2), pad_input=int(p.pad_input), cut_input=int(p.cut_input),
                k1=float(p.k1), k2=float(p.k2), m=int(p.m))


def _stream_handle(stream) -> int:
    import torch
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dev_words(t, nbits: int, name: str):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor of 64-bit words")
    if t.dtype not in (torch.int64, torch.uint64) or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous int64/uint64 tensor")
    if t.numel() < words(nbits):
        raise ValueError(f"{name} holds {t.numel()} words, needs {words(nbits)} for {nbits} bits")
    return t.data_ptr()


class Context:
    """A libcm context on one CUDA device."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0, max_transform_lg: int = 0, field: int = 0,
                 max_sum_blocks: int = 0, plan_mode: int = 0):
        import torch
        self.device = device
        torch.cuda.set_device(device)
        self._L = lib()
        opts = Options(hbm_budget_bytes, max_transform_lg, field, max_sum_blocks, plan_mode)
        h = ctypes.c_void_p()
        _check(self._L.cm_create(ctypes.byref(h), device, ctypes.byref(opts)), "cm_create")
        self._h = h

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            self._L.cm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _out(self, z, m, like):
        import torch
        if z is None:
            z = torch.empty(words(m), dtype=torch.int64, device=like.device)
        _dev_words(z, m, "z")
        return z

    def toeplitz(self, x, n: int, y, m: int, z=None, stream=None):
        """z = toep(y) x over GF(2): x has n bits, y has n + m - 1 bits."""
        px = _dev_words(x, n, "x")
        py = _dev_words(y, n + m - 1, "y")
        z = self._out(z, m, x)
        _check(self._L.cm_toeplitz(self._h, px, n, py, m, z.data_ptr(), _stream_handle(stream)),
               "cm_toeplitz")
        return z

    def circulant(self, x, n: int, y, m: int, z=None, stream=None):
        """Circulant(x, y): x has n bits, y has n + 1 bits (n + 1 prime in N_A)."""
        px = _dev_words(x, n, "x")
        py = _dev_words(y, n + 1, "y")
        z = self._out(z, m, x)
        _check(self._L.cm_circulant(self._h, px, n, py, m, z.data_ptr(), _stream_handle(stream)),
               "cm_circulant")
        return z

    def dodis(self, x, y, n: int, m: int, z=None, stream=None):
        """Dodis et al.(x, y): both n bits, n prime in N_A."""
        px = _dev_words(x, n, "x")
        py = _dev_words(y, n, "y")
        z = self._out(z, m, x)
        _check(self._L.cm_dodis(self._h, px, py, n, m, z.data_ptr(), _stream_handle(stream)),
               "cm_dodis")
        return z

    def compose(self, kind1: int, x, n1: int, y, m1: int, kind2: int, n2: int, m2: int, z=None, stream=None):
        """Composed extractor (cm_compose): s = Ext_kind1(x, y) (m1 bits), then
        t = Ext_kind2(first n2 bits of y, seed = first bits of s) (m2 bits);
        returns z = s followed by t (m1 + m2 bits)."""
        ybits = {TOEPLITZ: n1 + m1 - 1, CIRCULANT: n1 + 1, DODIS: n1}.get(kind1, 0)
        px = _dev_words(x, n1, "x")
        py = _dev_words(y, ybits, "y")
        z = self._out(z, m1 + m2, x)
        _check(self._L.cm_compose(self._h, kind1, px, n1, py, m1, kind2, n2, m2, z.data_ptr(),
                                  _stream_handle(stream)), "cm_compose")
        return z

    def calibrate(self, cache: str | None = None, force: bool = False, max_lg: int = 0):
        """Time the planner's figures on this GPU (cm_calibrate), or load them
        from `cache` when it matches the device."""
        _check(self._L.cm_calibrate(self._h, cache.encode() if cache else None, TUNE_FORCE if force else 0,
                                    max_lg), "cm_calibrate")

    def tune_query(self, field: int, lg: int) -> tuple[float, float, int]:
        """(ms, cluster_ms, split) of the calibration for field and 2^lg (0 where none)."""
        ms, cl, sp = ctypes.c_double(0), ctypes.c_double(0), ctypes.c_int32(0)
        _check(self._L.cm_tune_query(self._h, field, lg, ctypes.byref(ms), ctypes.byref(cl), ctypes.byref(sp)),
               "cm_tune_query")
        return ms.value, cl.value, sp.value

    def von_neumann(self, x, n: int, z=None, m_out=None, stream=None):
        """Von Neumann extraction on the device (cm_von_neumann).  Returns
        (z, m_out): z has room for the longest output, m_out is a one-element
        device tensor that receives the output length."""
        import torch
        px = _dev_words(x, n, "x")
        if z is None:
            z = torch.empty(max(1, words(n // 2)), dtype=torch.int64, device=x.device)
        pz = _dev_words(z, n // 2, "z")
        if m_out is None:
            m_out = torch.zeros(1, dtype=torch.int64, device=x.device)
        pm = _dev_words(m_out, 64, "m_out")
        _check(self._L.cm_von_neumann(self._h, px, n, pz, pm, _stream_handle(stream)), "cm_von_neumann")
        return z, m_out

    def trevisan_rsh(self, x, n: int, l: int, seeds, m: int, z=None, stream=None):
        """m RSH one-bit extractions of x; one-bit seed i = bits 2 l i .. 2 l i + 2l - 1 of seeds."""
        _dev_words(x, n, "x")
        _dev_words(seeds, 2 * l * m, "seeds")
        z = self._out(z, m, x)
        _check(self._L.cm_trevisan_rsh(self._h, x.data_ptr(), n, l, seeds.data_ptr(), m, z.data_ptr(),
                                       _stream_handle(stream)), "cm_trevisan_rsh")
        return z

    def trevisan(self, x, n: int, y, d: int, sets, t: int, m: int, l: int, z=None, stream=None):
        """Trevisan(x, y) over the weak design's sets (m x t uint32 / int32 device array)."""
        _dev_words(x, n, "x")
        _dev_words(y, d, "y")
        if sets.device.type != "cuda" or sets.numel() < m * t or sets.element_size() != 4:
            raise ValueError("sets: a CUDA tensor of m * t 32-bit indices")
        z = self._out(z, m, x)
        _check(self._L.cm_trevisan(self._h, x.data_ptr(), n, y.data_ptr(), d, sets.data_ptr(), t, m, l,
                                   z.data_ptr(), _stream_handle(stream)), "cm_trevisan")
        return z

    def von_neumann_host(self, x, n: int, z, stream=None) -> tuple[int, int]:
        """End-to-end Von Neumann on host tensors; returns (cm_status, m)."""
        for t, nb, nm in ((x, n, "x"), (z, n // 2, "z")):
            if t.is_cuda or t.numel() < words(nb) or t.element_size() != 8 or not t.is_contiguous():
                raise ValueError(f"{nm} must be a contiguous host tensor of >= {words(nb)} words")
        m = _U64(0)
        s = self._L.cm_von_neumann_host(self._h, x.data_ptr(), n, z.data_ptr(), ctypes.byref(m),
                                        _stream_handle(stream))
        if s not in (CM_OK, CM_EPRECOND):
            raise CMError(s, "cm_von_neumann_host")
        return int(s), int(m.value)

    def extract_host(self, kind: int, x, n: int, y, m: int, z, stream=None) -> int:
        """End-to-end call on host buffers (torch CPU tensors, ideally pinned):
        host->device copies, extraction, device->host copy, stream sync.
        Returns the cm_status (CM_EPRECOND for a constant Dodis et al. x)."""
        ybits = n + m - 1 if kind == TOEPLITZ else (n + 1 if kind == CIRCULANT else n)
        for t, nb, nm in ((x, n, "x"), (y, ybits, "y"), (z, m, "z")):
            if t.is_cuda or t.numel() < words(nb) or t.element_size() != 8 or not t.is_contiguous():
                raise ValueError(f"{nm} must be a contiguous host tensor of >= {words(nb)} words")
        s = self._L.cm_extract_host(self._h, kind, x.data_ptr(), n, y.data_ptr(), m, z.data_ptr(),
                                    _stream_handle(stream))
        if s not in (CM_OK, CM_EPRECOND):
            raise CMError(s, "cm_extract_host")
        return int(s)

    def profile_enable(self, on: bool = True):
        _check(self._L.cm_profile_enable(self._h, 1 if on else 0), "cm_profile_enable")

    def profile_read(self, reset: bool = True) -> dict:
        """{kernel name: (launches, total_ms)} for traced launches."""
        cap = 64
        buf = (ProfileEntry * cap)()
        cnt = ctypes.c_uint32(0)
        _check(self._L.cm_profile_read(self._h, ctypes.cast(buf, ctypes.c_void_p), cap,
                                       ctypes.byref(cnt), 1 if reset else 0), "cm_profile_read")
        return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].total_ms))
                for i in range(min(cap, cnt.value))}

    @staticmethod
    def _descs(items):
        """items: (kind, n, m, x, y, z) with x, y, z CUDA word tensors."""
        arr = (CmDesc * max(1, len(items)))()
        for i, (kind, n, m, x, y, z) in enumerate(items):
            ybits = n + m - 1 if kind == TOEPLITZ else (n + 1 if kind == CIRCULANT else n)
            arr[i] = CmDesc(kind, 0, n, m, _dev_words(x, n, "x"), _dev_words(y, ybits, "y"),
                            _dev_words(z, m, "z"))
        return arr

    def batch(self, items, autotune: bool = False, graph: bool = True, test_stall: bool = False) -> "Batch":
        """Plan a batch (cm_batch_create); items are (kind, n, m, x, y, z)."""
        arr = self._descs(items)
        flags = (BATCH_AUTOTUNE if autotune else 0) | (0 if graph else BATCH_NO_GRAPH)
        flags |= BATCH_TEST_STALL if test_stall else 0
        h = ctypes.c_void_p()
        _check(self._L.cm_batch_create(self._h, ctypes.cast(arr, ctypes.c_void_p), len(items), flags,
                                       ctypes.byref(h)), "cm_batch_create")
        return Batch(self, h, items)

    def batch_extract(self, items, stream=None):
        """One-shot batch (cm_batch_extract): returns after the outputs are written."""
        arr = self._descs(items)
        _check(self._L.cm_batch_extract(self._h, ctypes.cast(arr, ctypes.c_void_p), len(items),
                                        _stream_handle(stream)), "cm_batch_extract")

    def toeplitz_shared_seed(self, y, n: int, m: int, X, count: int, Z=None, engine: int = ENGINE_AUTO,
                             stream=None):
        """count Toeplitz extractions under one seed y: X holds the inputs back to
        back (ceil(n/64) words each); returns Z (ceil(m/64) words each)."""
        import torch
        py = _dev_words(y, n + m - 1, "y")
        pX = _dev_words(X, words(n) * 64 * count, "X")
        if Z is None:
            Z = torch.empty(words(m) * count, dtype=torch.int64, device=X.device)
        _dev_words(Z, words(m) * 64 * count, "Z")
        _check(self._L.cm_batch_toeplitz_shared_seed(self._h, py, n, m, pX, count, Z.data_ptr(), engine,
                                                     _stream_handle(stream)), "cm_batch_toeplitz_shared_seed")
        return Z

    # ----- serving -------------------------------------------------------------
    def server_start(self, hbm_budget_bytes: int = 0, slots: int = 0, max_queue: int = 0, max_wave: int = 0,
                     seed_cache_bytes: int = 0, express_slots: int = 0):
        """express_slots: 0 = one, SERVER_NO_EXPRESS = none."""
        o = ServerOptions(hbm_budget_bytes, slots, max_queue, max_wave, express_slots, seed_cache_bytes)
        _check(self._L.cm_server_start(self._h, ctypes.byref(o)), "cm_server_start")

    def server_stop(self):
        _check(self._L.cm_server_stop(self._h), "cm_server_stop")

    def submit_raw(self, kind: int, n: int, m: int, px: int, py: int, pz: int, seed_id: int = 0) -> tuple[int, int]:
        """(status, ticket) for device pointers; no exception on CM_EAGAIN / CM_ENOMEM.
        seed_id != 0 asks the server to keep the seed's transform resident."""
        r = CmRequest(kind, REQ_SEED_CACHE if seed_id else 0, n, m, px, py, pz, seed_id, 0)
        t = ctypes.c_uint64(0)
        s = self._L.cm_submit(self._h, ctypes.byref(r), ctypes.byref(t))
        return int(s), int(t.value)

    def submit(self, kind: int, n: int, m: int, x, y, z, seed_id: int = 0) -> int:
        ybits = n + m - 1 if kind == TOEPLITZ else (n + 1 if kind == CIRCULANT else n)
        s, t = self.submit_raw(kind, n, m, _dev_words(x, n, "x"), _dev_words(y, ybits, "y"),
                               _dev_words(z, m, "z"), seed_id)
        _check(s, "cm_submit")
        return t

    def poll(self, ticket: int, timeout_s: float = 0.0):
        """(cm_status of the poll, result dict or None)."""
        r = CmResult()
        s = self._L.cm_poll(self._h, ticket, ctypes.byref(r), int(timeout_s * 1e9))
        if s != CM_OK:
            return int(s), None
        return CM_OK, {k: getattr(r, k) for k, _ in CmResult._fields_}

    def server_stats(self) -> dict:
        st = ServerStats()
        _check(self._L.cm_server_get_stats(self._h, ctypes.byref(st)), "cm_server_get_stats")
        return {k: getattr(st, k) for k, _ in ServerStats._fields_ if k != "reserved"}

    def device_status(self, stream=None) -> tuple[int, int]:
        f = ctypes.c_uint32(0)
        s = self._L.cm_device_status(self._h, _stream_handle(stream), ctypes.byref(f))
        return int(s), int(f.value)


class Batch:
    """A planned batch (cm_batch); keeps its descriptors' tensors alive."""

    def __init__(self, ctx: Context, handle, items):
        self._ctx = ctx
        self._h = handle
        self._items = items

    def launch(self, stream=None):
        _check(self._ctx._L.cm_batch_launch(self._h, _stream_handle(stream)), "cm_batch_launch")

    def info(self) -> dict:
        st = BatchStats()
        _check(self._ctx._L.cm_batch_info(self._h, ctypes.byref(st)), "cm_batch_info")
        return {k: getattr(st, k) for k, _ in BatchStats._fields_}

    def close(self):
        if getattr(self, "_h", None):
            self._ctx._L.cm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

"""Thin Python binding of the C ABI in ``include/lbm.h`` (ctypes).

Argument marshalling only: every step of the method runs in the CUDA kernels of
``liblbm_gb300.so``. PyTorch supplies device memory (the simulation's arena is a
torch uint8 tensor) and the CUDA stream (the current torch stream at creation).
If the library is missing or no GPU is usable the calls raise; there is no
fallback.

Functions carry the C names (``lbm_create``, ``lbm_step``, ``lbm_front_heights``,
``lbm_fields`` ...); ``Simulation`` wraps one handle.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbm_gb300.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "lbm.h")

GROWTH_MODES = {"none": 0, "bulk": 1, "density": 2, "edge": 3, "band": 4}
FRONT_KINDS = {"flat": 0, "sinusoidal": 1, "full": 2}
WALL_MODES = {"fixed": 0, "advance": 1}
NEGFIX_MODES = {"literal": 0, "rescale": 1}
PRECISIONS = {"fp32": 0, "fp64": 1, "fp16": 2, "bf16": 3}

LBM_OK = 0
STATUS_FRONT_AT_TOP = 1
STATUS_GROWTH_STARVED = 2
STATUS_CAPACITY = 4
STATUS_TIMEOUT = 8
LATTICES = {"d2q9": 0, "d2q7": 1}
UPDATE_KERNELS = {"auto": 0, "plain": 1, "tma": 2, "tma1": 3, "tma_sel": 4, "shared": 5, "tma_st": 6}


class LbmError(RuntimeError):
    pass


class lbm_params_t(ctypes.Structure):
    _fields_ = [
        ("tau", ctypes.c_double), ("mu", ctypes.c_double), ("rho_c", ctypes.c_double),
        ("rho_cell", ctypes.c_double), ("sigma", ctypes.c_double), ("rho0", ctypes.c_double),
        ("growth_rate", ctypes.c_double), ("rho_init", ctypes.c_double),
        ("rho_jitter", ctypes.c_double), ("front_row", ctypes.c_double),
        ("front_amp", ctypes.c_double), ("wall_min_gap", ctypes.c_double),
        ("wall_w_factor", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("width", ctypes.c_int32), ("height", ctypes.c_int32), ("growth_mode", ctypes.c_int32),
        ("edge_depth", ctypes.c_int32), ("band_rows", ctypes.c_int32),
        ("front_kind", ctypes.c_int32), ("front_kmin", ctypes.c_int32),
        ("front_kmax", ctypes.c_int32), ("wall_mode", ctypes.c_int32),
        ("negfix_mode", ctypes.c_int32), ("y_periodic", ctypes.c_int32),
        ("sim_id", ctypes.c_uint32), ("precision", ctypes.c_int32), ("update_kernel", ctypes.c_int32),
        ("lattice", ctypes.c_int32), ("plan_blocks", ctypes.c_int32),
    ]


class lbm_stats_t(ctypes.Structure):
    _fields_ = [
        ("step", ctypes.c_int64), ("ns_last", ctypes.c_int64), ("ns_total", ctypes.c_int64),
        ("div_total", ctypes.c_int64), ("starved_steps", ctypes.c_int64),
        ("cand_last", ctypes.c_int64), ("events_last", ctypes.c_int64),
        ("mass_fix", ctypes.c_int64), ("quiescent_fix", ctypes.c_int64),
        ("S1", ctypes.c_int64), ("S2", ctypes.c_int64), ("node_updates", ctypes.c_int64),
        ("launches", ctypes.c_int64),
        ("mass", ctypes.c_double), ("quiescent_mass", ctypes.c_double),
        ("carry", ctypes.c_double), ("hbar", ctypes.c_double), ("w", ctypes.c_double),
        ("clip_mass", ctypes.c_double),
        ("y_r", ctypes.c_int32), ("H_top", ctypes.c_int32), ("hmin", ctypes.c_int32),
        ("y_hi", ctypes.c_int32), ("status", ctypes.c_int32), ("update_kernel", ctypes.c_int32),
    ]


_P = ctypes.c_void_p
_SIGNATURES = {
    "lbm_validate": (ctypes.c_int, [ctypes.POINTER(lbm_params_t)]),
    "lbm_footprint": (ctypes.c_int, [ctypes.POINTER(lbm_params_t), ctypes.POINTER(ctypes.c_uint64)]),
    "lbm_plan_capacity": (ctypes.c_int, [ctypes.POINTER(lbm_params_t), ctypes.POINTER(ctypes.c_int64)]),
    "lbm_front_heights_async": (ctypes.c_int, [_P, _P, _P]),
    "lbm_eq6": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(ctypes.c_double),
                               ctypes.POINTER(ctypes.c_double)]),
    "lbm_eq6_n": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int32, _P, _P]),
    "lbm_create": (ctypes.c_int, [ctypes.POINTER(lbm_params_t), _P, _P, ctypes.c_uint64,
                                  ctypes.POINTER(_P)]),
    "lbm_step": (ctypes.c_int, [_P, ctypes.c_int64]),
    "lbm_front_heights": (ctypes.c_int, [_P, _P, _P, _P]),
    "lbm_fields": (ctypes.c_int, [_P, _P, _P, _P]),
    "lbm_fields_device": (ctypes.c_int, [_P, _P, _P, _P]),
    "lbm_populations": (ctypes.c_int, [_P, _P]),
    "lbm_set_populations": (ctypes.c_int, [_P, _P]),
    "lbm_mask": (ctypes.c_int, [_P, _P]),
    "lbm_last_events": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int64, _P]),
    "lbm_stats": (ctypes.c_int, [_P, ctypes.POINTER(lbm_stats_t)]),
    "lbm_clear_status": (ctypes.c_int, [_P]),
    "lbm_debug_waits": (ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_int32]),
    "lbm_timing_enable": (ctypes.c_int, [_P, ctypes.c_int64]),
    "lbm_timing_read": (ctypes.c_int, [_P, _P, _P, _P]),
    "lbm_timing_stride": (ctypes.c_int, [_P, ctypes.c_int64]),
    "lbm_bytes_per_node": (ctypes.c_int, [_P, _P]),
    "lbm_sync": (ctypes.c_int, [_P]),
    "lbm_destroy": (None, [_P]),
    "lbm_strerror": (ctypes.c_char_p, [ctypes.c_int]),
    "lbm_last_cuda_error": (ctypes.c_char_p, []),
    "lbm_version": (ctypes.c_char_p, []),
    "lbm_front_heights_noalloc": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, _P, _P, _P]),
    "lbm_batch_create": (ctypes.c_int, [_P, ctypes.c_int32, _P, ctypes.POINTER(_P)]),
    "lbm_batch_step": (ctypes.c_int, [_P, ctypes.c_int64]),
    "lbm_batch_destroy": (ctypes.c_int, [_P]),
    "lbm_batch_fused": (ctypes.c_int, [_P]),
    "lbm_batch_create_empty": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P,
                                              ctypes.POINTER(_P)]),
    "lbm_batch_attach": (ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_int32)]),
    "lbm_batch_detach": (ctypes.c_int, [_P, _P]),
    "lbm_batch_members": (ctypes.c_int, [_P]),
    "lbm_batch_captures": (ctypes.c_int, [_P]),
}

_lib = None


def header_functions(path: str = HEADER):
    """Names of the functions declared in ``include/lbm.h``."""
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_0-9]+)\s*\(", text)))


def load_library(path: str = LIB_PATH):
    """Loads ``liblbm_gb300.so`` (building it first if it is absent); raises if
    it cannot be loaded."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            from . import build as _build
            _build.build()
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(rc: int, what: str):
    if rc != LBM_OK:
        lib = load_library()
        msg = lib.lbm_strerror(rc).decode()
        if rc == -3 or rc == -2 or rc == -5:
            msg += " (" + lib.lbm_last_cuda_error().decode() + ")"
        raise LbmError(f"{what}: {msg} [{rc}]")


def make_params(d: dict, precision: str = "fp32", update_kernel: str = "auto") -> lbm_params_t:
    p = lbm_params_t()
    for name, _ in lbm_params_t._fields_:
        if name == "precision":
            v = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        elif name == "update_kernel":
            v = UPDATE_KERNELS[update_kernel] if isinstance(update_kernel, str) else int(update_kernel)
        elif name == "lattice":
            v = d.get("lattice", "d2q9")
            v = LATTICES[v] if isinstance(v, str) else int(v)
        elif name == "plan_blocks":
            v = int(d.get("plan_blocks", 0))
        else:
            v = d[name]
            if name == "growth_mode" and isinstance(v, str):
                v = GROWTH_MODES[v]
            elif name == "front_kind" and isinstance(v, str):
                v = FRONT_KINDS[v]
            elif name == "wall_mode" and isinstance(v, str):
                v = WALL_MODES[v]
            elif name == "negfix_mode" and isinstance(v, str):
                v = NEGFIX_MODES[v]
        setattr(p, name, v)
    return p


def lbm_validate(params: dict, precision: str = "fp32") -> int:
    p = make_params(params, precision)
    return load_library().lbm_validate(ctypes.byref(p))


def lbm_plan_capacity(params: dict, precision: str = "fp32") -> int:
    """Divisions per step the planner of such a simulation holds."""
    p = make_params(params, precision)
    out = ctypes.c_int64()
    _check(load_library().lbm_plan_capacity(ctypes.byref(p), ctypes.byref(out)), "lbm_plan_capacity")
    return int(out.value)


def lbm_footprint(params: dict, precision: str = "fp32") -> int:
    p = make_params(params, precision)
    out = ctypes.c_uint64()
    _check(load_library().lbm_footprint(ctypes.byref(p), ctypes.byref(out)), "lbm_footprint")
    return int(out.value)


def lbm_eq6(s1: int, s2: int, width: int):
    """Eq. 6 (hbar, w) from the exact sums of the front heights."""
    hbar, w = ctypes.c_double(), ctypes.c_double()
    _check(load_library().lbm_eq6(int(s1), int(s2), int(width), ctypes.byref(hbar), ctypes.byref(w)), "lbm_eq6")
    return hbar.value, w.value


def lbm_eq6_n(sums, width: int):
    """Eq. 6 for n (S1, S2) pairs: `sums` is a host int64 array or CPU tensor
    of shape (n, 2) (the layout lbm_front_heights_async writes); returns
    float64 arrays (hbar, w) of length n, each pair as lbm_eq6 gives it."""
    import numpy as np
    a = np.ascontiguousarray(sums.numpy() if hasattr(sums, "numpy") else sums, dtype=np.int64).reshape(-1, 2)
    n = a.shape[0]
    hbar = np.empty(n, dtype=np.float64)
    w = np.empty(n, dtype=np.float64)
    _check(load_library().lbm_eq6_n(_P(a.ctypes.data), n, int(width), _P(hbar.ctypes.data), _P(w.ctypes.data)),
           "lbm_eq6_n")
    return hbar, w


def lbm_front_heights_noalloc(mask_dev, width: int, height: int, heights_dev, stats_dev, stream=None):
    """Allocation-free front heights and width of a device occupancy bitmask
    (``include/lbm.h``). ``mask_dev`` (uint32, H x ceil(W/32)), ``heights_dev``
    (int32, W) and ``stats_dev`` (float64, 2) are torch CUDA tensors owned by
    the caller; nothing is allocated. Enqueued on ``stream`` (default: the
    current torch stream)."""
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    _check(load_library().lbm_front_heights_noalloc(
        ctypes.c_void_p(mask_dev.data_ptr()), int(width), int(height), ctypes.c_void_p(heights_dev.data_ptr()),
        ctypes.c_void_p(stats_dev.data_ptr()), ctypes.c_void_p(s.cuda_stream)), "lbm_front_heights_noalloc")


class Simulation:
    """One resident simulation (``lbm_create`` ... ``lbm_destroy``)."""

    def __init__(self, params: dict, precision: str = "fp32", device=None, stream=None,
                 update_kernel: str = "auto"):
        import torch
        lib = load_library()
        if not torch.cuda.is_available():
            raise LbmError("lbm_create: no CUDA device")
        self.params = dict(params)
        self.precision = precision
        self.W = int(params["width"])
        self.H = int(params["height"])
        self.Q = 7 if params.get("lattice", "d2q9") in ("d2q7", 1) else 9  # population planes
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self._p = make_params(params, precision, update_kernel)
        nbytes = lbm_footprint(params, precision)
        with torch.cuda.device(self.device):
            self.stream = torch.cuda.current_stream(self.device) if stream is None else stream
            # the arena is torch-owned device memory, kept alive by this object
            self.arena = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
            base = self.arena.data_ptr()
            aligned = (base + 255) & ~255
            h = ctypes.c_void_p()
            _check(lib.lbm_create(ctypes.byref(self._p), ctypes.c_void_p(self.stream.cuda_stream),
                                  ctypes.c_void_p(aligned), nbytes, ctypes.byref(h)), "lbm_create")
        self._h = h
        self._lib = lib

    # -- life cycle
    def close(self):
        if getattr(self, "_h", None):
            self._lib.lbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- C ABI
    def lbm_step(self, n: int = 1):
        _check(self._lib.lbm_step(self._h, int(n)), "lbm_step")

    step = lbm_step

    def lbm_front_heights_async(self, h_pinned, sums_pinned):
        """Enqueues the copies of h(x) and of the Eq. 6 sums (S1, S2) into
        caller-owned pinned torch CPU tensors (int32 W, int64 2); valid after
        ``sync()``. ``h_pinned`` may be None."""
        _check(self._lib.lbm_front_heights_async(
            self._h, None if h_pinned is None else ctypes.c_void_p(h_pinned.data_ptr()),
            ctypes.c_void_p(sums_pinned.data_ptr())), "lbm_front_heights_async")

    def lbm_front_heights(self):
        h = np.empty(self.W, dtype=np.int32)
        hbar = ctypes.c_double()
        w = ctypes.c_double()
        _check(self._lib.lbm_front_heights(self._h, h.ctypes.data, ctypes.byref(hbar), ctypes.byref(w)),
               "lbm_front_heights")
        return h, hbar.value, w.value

    front_heights = lbm_front_heights

    def lbm_fields(self):
        rho = np.empty((self.H, self.W))
        ux = np.empty((self.H, self.W))
        uy = np.empty((self.H, self.W))
        _check(self._lib.lbm_fields(self._h, rho.ctypes.data, ux.ctypes.data, uy.ctypes.data), "lbm_fields")
        return rho, ux, uy

    fields = lbm_fields

    def lbm_fields_device(self, rho, ux, uy):
        """Writes into three caller-owned torch float64 CUDA tensors of H*W."""
        _check(self._lib.lbm_fields_device(self._h, ctypes.c_void_p(rho.data_ptr()),
                                           ctypes.c_void_p(ux.data_ptr()), ctypes.c_void_p(uy.data_ptr())),
               "lbm_fields_device")

    def lbm_populations(self):
        f = np.empty((self.Q, self.H, self.W))
        _check(self._lib.lbm_populations(self._h, f.ctypes.data), "lbm_populations")
        return f

    pops = lbm_populations

    def lbm_set_populations(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        assert f.shape == (self.Q, self.H, self.W)
        _check(self._lib.lbm_set_populations(self._h, f.ctypes.data), "lbm_set_populations")

    set_pops = lbm_set_populations

    def lbm_mask(self):
        m = np.empty((self.H, self.W), dtype=np.uint8)
        _check(self._lib.lbm_mask(self._h, m.ctypes.data), "lbm_mask")
        return m.astype(bool)

    mask = lbm_mask

    def heights(self):
        return self.lbm_front_heights()[0]

    def lbm_last_events(self):
        n = ctypes.c_int64()
        _check(self._lib.lbm_last_events(self._h, None, None, None, 0, ctypes.byref(n)), "lbm_last_events")
        k = max(n.value, 1)
        node = np.empty(k, dtype=np.int64)
        pair = np.empty(k, dtype=np.int32)
        cnt = np.empty(k, dtype=np.int32)
        _check(self._lib.lbm_last_events(self._h, node.ctypes.data, pair.ctypes.data, cnt.ctypes.data,
                                         n.value, ctypes.byref(n)), "lbm_last_events")
        return node[:n.value], pair[:n.value], cnt[:n.value]

    last_events = lbm_last_events

    def lbm_stats(self) -> dict:
        s = lbm_stats_t()
        _check(self._lib.lbm_stats(self._h, ctypes.byref(s)), "lbm_stats")
        return {name: getattr(s, name) for name, _ in lbm_stats_t._fields_}

    stats = lbm_stats

    def lbm_clear_status(self):
        _check(self._lib.lbm_clear_status(self._h), "lbm_clear_status")

    def lbm_debug_waits(self, budget_cycles: int = 0, withhold: int = 0):
        """Failure-detection test hook: wait budget in clock cycles (0: the
        default) and what is withheld (bit 0 bulk copies, bit 1 one grid-
        barrier arrival) so that the bounded waits run out."""
        _check(self._lib.lbm_debug_waits(self._h, int(budget_cycles), int(withhold)), "lbm_debug_waits")

    def lbm_timing_enable(self, max_launches: int):
        _check(self._lib.lbm_timing_enable(self._h, int(max_launches)), "lbm_timing_enable")

    def lbm_timing_stride(self, stride: int):
        _check(self._lib.lbm_timing_stride(self._h, int(stride)), "lbm_timing_stride")

    def lbm_timing_read(self):
        n = ctypes.c_int64()
        ms = ctypes.c_double()
        nodes = ctypes.c_int64()
        _check(self._lib.lbm_timing_read(self._h, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(nodes)),
               "lbm_timing_read")
        return n.value, ms.value, nodes.value

    def lbm_bytes_per_node(self) -> int:
        b = ctypes.c_int64()
        _check(self._lib.lbm_bytes_per_node(self._h, ctypes.byref(b)), "lbm_bytes_per_node")
        return b.value

    def lbm_sync(self):
        _check(self._lib.lbm_sync(self._h), "lbm_sync")

    sync = lbm_sync


class Batch:
    """Independent simulations stepped together (``lbm_batch_create`` ...
    ``lbm_batch_destroy``): one CUDA-graph replay advances every member, the
    members' kernels running side by side. Keeps the members alive.

    ``Batch.empty(slots, precision, lattice)`` makes a batch with free slots
    (``lbm_batch_create_empty``); ``attach``/``detach`` let members join and
    leave it without capturing its graphs again."""

    def __init__(self, sims, stream=None):
        import torch
        lib = load_library()
        self.sims = list(sims)
        if not self.sims:
            raise LbmError("lbm_batch_create: no simulations")
        self._lib = lib
        dev = self.sims[0].device
        with torch.cuda.device(dev):
            self.stream = torch.cuda.current_stream(dev) if stream is None else stream
            arr = (_P * len(self.sims))(*[s._h.value for s in self.sims])
            h = _P()
            _check(lib.lbm_batch_create(ctypes.cast(arr, _P), len(self.sims), _P(self.stream.cuda_stream),
                                        ctypes.byref(h)), "lbm_batch_create")
        self._h = h

    @classmethod
    def empty(cls, slots: int, precision: str = "fp32", lattice: str = "d2q9", device: int = 0, stream=None):
        """A batch with `slots` free slots for simulations of one lattice and
        storage type on `device`."""
        import torch
        self = cls.__new__(cls)
        self._lib = lib = load_library()
        self.sims = []
        with torch.cuda.device(device):
            self.stream = torch.cuda.current_stream(device) if stream is None else stream
            h = _P()
            _check(lib.lbm_batch_create_empty(int(slots), LATTICES[lattice], PRECISIONS[precision],
                                              _P(self.stream.cuda_stream), ctypes.byref(h)),
                   "lbm_batch_create_empty")
        self._h = h
        return self

    def attach(self, sim) -> int:
        """Puts `sim` into a free slot and returns the slot's index; raises
        LbmError if none is free (LBM_ERR_BATCH_FULL) or `sim` does not fit
        the batch."""
        slot = ctypes.c_int32(-1)
        _check(self._lib.lbm_batch_attach(self._h, sim._h, ctypes.byref(slot)), "lbm_batch_attach")
        self.sims.append(sim)
        return slot.value

    def detach(self, sim):
        _check(self._lib.lbm_batch_detach(self._h, sim._h), "lbm_batch_detach")
        self.sims = [s for s in self.sims if s is not sim]

    @property
    def members(self) -> int:
        return self._lib.lbm_batch_members(self._h)

    @property
    def captures(self) -> int:
        """How many times the batch's graphs were captured (1 after creation)."""
        return self._lib.lbm_batch_captures(self._h)

    def lbm_batch_step(self, n: int = 1):
        _check(self._lib.lbm_batch_step(self._h, int(n)), "lbm_batch_step")

    step = lbm_batch_step

    @property
    def fused(self) -> bool:
        """True if a step of the batch is three batched launches."""
        return self._lib.lbm_batch_fused(self._h) >= 1

    @property
    def staged(self) -> bool:
        """True if the batched update is the TMA-staged one."""
        return self._lib.lbm_batch_fused(self._h) >= 2

    @property
    def bulk_stores(self) -> bool:
        """True if the staged batched update stores by bulk tensor copies."""
        return self._lib.lbm_batch_fused(self._h) == 3

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lbm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

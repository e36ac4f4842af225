"""Python wrapper (ctypes) around the plain FP64 CPU oracle in ``lbm_oracle.c``.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers. The product path never
imports this module. It shares no code with the CUDA library: it takes the same
plain parameter dictionary (see ``paper_2303_02210_gb300/workloads.py``) and
marshals it into its own C struct.

The oracle restates App. A of Killeen et al. (arXiv 2303.02210) step by step,
over the whole lattice, in IEEE double with no fused multiply-add; see the
header of ``lbm_oracle.c`` for the readings it takes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB = os.path.join(_HERE, "liblbm_oracle.so")

GROWTH_MODES = {"none": 0, "bulk": 1, "density": 2, "edge": 3, "band": 4}
FRONT_KINDS = {"flat": 0, "sinusoidal": 1, "full": 2}
WALL_MODES = {"fixed": 0, "advance": 1}
NEGFIX_MODES = {"literal": 0, "rescale": 1}
LATTICES = {"d2q9": 0, "d2q7": 1}


class _Params(ctypes.Structure):
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
        ("sim_id", ctypes.c_uint32),
        ("lattice", ctypes.c_int32),
    ]


class _Stats(ctypes.Structure):
    _fields_ = [
        ("step", ctypes.c_int64), ("ns_last", ctypes.c_int64), ("ns_total", ctypes.c_int64),
        ("div_total", ctypes.c_int64), ("starved_steps", ctypes.c_int64),
        ("cand_last", ctypes.c_int64), ("events_last", ctypes.c_int64),
        ("mass_fix", ctypes.c_int64), ("quiescent_fix", ctypes.c_int64),
        ("S1", ctypes.c_int64), ("S2", ctypes.c_int64),
        ("mass", ctypes.c_double), ("quiescent_mass", ctypes.c_double),
        ("carry", ctypes.c_double), ("hbar", ctypes.c_double), ("w", ctypes.c_double),
        ("clip_mass", ctypes.c_double),
        ("y_r", ctypes.c_int32), ("H_top", ctypes.c_int32), ("hmin", ctypes.c_int32),
        ("status", ctypes.c_int32),
    ]


def build_oracle(force: bool = False) -> str:
    """Compile ``lbm_oracle.c`` into ``liblbm_oracle.so`` (gcc, no FMA contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_oracle())
        lib.orc_create.restype = ctypes.c_void_p
        lib.orc_create.argtypes = [ctypes.POINTER(_Params)]
        lib.orc_destroy.argtypes = [ctypes.c_void_p]
        lib.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_int64]
        for name in ("orc_get_pops", "orc_set_pops"):
            getattr(lib, name).argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        lib.orc_get_mask.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        lib.orc_get_heights.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
        lib.orc_get_stats.argtypes = [ctypes.c_void_p, ctypes.POINTER(_Stats)]
        lib.orc_fields.argtypes = [ctypes.c_void_p] * 4
        lib.orc_last_events.restype = ctypes.c_int64
        lib.orc_last_events.argtypes = [ctypes.c_void_p] * 4 + [ctypes.c_int64]
        lib.orc_philox4x32_10.argtypes = [ctypes.c_void_p] * 3
        lib.orc_sizeof_params.restype = ctypes.c_int32
        lib.orc_sizeof_stats.restype = ctypes.c_int32
        lib.orc_directions.restype = ctypes.c_int32
        lib.orc_directions.argtypes = [ctypes.c_void_p]
        assert lib.orc_sizeof_params() == ctypes.sizeof(_Params)
        assert lib.orc_sizeof_stats() == ctypes.sizeof(_Stats)
        _lib = lib
    return _lib


def _params(d: dict) -> _Params:
    p = _Params()
    for name, ctype in _Params._fields_:
        v = d.get(name, "d2q9") if name == "lattice" else d[name]
        if name == "growth_mode":
            v = GROWTH_MODES[v] if isinstance(v, str) else v
        elif name == "front_kind":
            v = FRONT_KINDS[v] if isinstance(v, str) else v
        elif name == "wall_mode":
            v = WALL_MODES[v] if isinstance(v, str) else v
        elif name == "negfix_mode":
            v = NEGFIX_MODES[v] if isinstance(v, str) else v
        elif name == "lattice":
            v = LATTICES[v] if isinstance(v, str) else v
        setattr(p, name, v)
    return p


def philox4x32_10(ctr, key):
    """Philox4x32-10 block: four 32-bit counter words, two key words -> four words."""
    lib = _load()
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib.orc_philox4x32_10(c, k, o)
    return tuple(int(v) for v in o)


class OracleSim:
    """One simulation held by the C oracle (FP64, dense over the lattice)."""

    def __init__(self, params: dict):
        self._lib = _load()
        self.params = dict(params)
        self.W = int(params["width"])
        self.H = int(params["height"])
        self._p = _params(params)
        self._h = self._lib.orc_create(ctypes.byref(self._p))
        if not self._h:
            raise ValueError("oracle rejected the parameters")
        self.Q = int(self._lib.orc_directions(self._h))

    def close(self):
        if self._h:
            self._lib.orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int = 1):
        self._lib.orc_step(self._h, int(n))

    def pops(self) -> np.ndarray:
        out = np.empty((self.Q, self.H, self.W), dtype=np.float64)
        self._lib.orc_get_pops(self._h, out.ctypes.data)
        return out

    def set_pops(self, f: np.ndarray):
        f = np.ascontiguousarray(f, dtype=np.float64)
        assert f.shape == (self.Q, self.H, self.W)
        self._lib.orc_set_pops(self._h, f.ctypes.data)

    def mask(self) -> np.ndarray:
        out = np.empty((self.H, self.W), dtype=np.uint8)
        self._lib.orc_get_mask(self._h, out.ctypes.data)
        return out.astype(bool)

    def heights(self) -> np.ndarray:
        out = np.empty(self.W, dtype=np.int32)
        self._lib.orc_get_heights(self._h, out.ctypes.data)
        return out

    def stats(self) -> dict:
        s = _Stats()
        self._lib.orc_get_stats(self._h, ctypes.byref(s))
        return {name: getattr(s, name) for name, _ in _Stats._fields_}

    def fields(self):
        rho = np.empty((self.H, self.W))
        ux = np.empty((self.H, self.W))
        uy = np.empty((self.H, self.W))
        self._lib.orc_fields(self._h, rho.ctypes.data, ux.ctypes.data, uy.ctypes.data)
        return rho, ux, uy

    def last_events(self):
        """(node, pair, count) of the divisions applied in the last step."""
        n = self._lib.orc_last_events(self._h, None, None, None, 0)
        node = np.empty(max(n, 1), dtype=np.int64)
        pair = np.empty(max(n, 1), dtype=np.int32)
        cnt = np.empty(max(n, 1), dtype=np.int32)
        self._lib.orc_last_events(self._h, node.ctypes.data, pair.ctypes.data,
                                  cnt.ctypes.data, n)
        return node[:n], pair[:n], cnt[:n]

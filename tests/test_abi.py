"""The C-ABI library loads, exports every function declared in include/lbm.h,
and its host-only logic (parameter checks, footprint, error strings) works
without a GPU. No compute call is made here."""
import ctypes

import numpy as np

import pytest

from paper_2303_02210_gb300 import lbm
from paper_2303_02210_gb300 import workloads as wl


@pytest.fixture(scope="module")
def lib():
    return lbm.load_library()


def test_exports_every_declared_function(lib):
    names = lbm.header_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(lbm._SIGNATURES), "binding and header disagree"


def test_struct_layouts_match_header():
    # 13 doubles, 1 uint64, 15 int32 words, padded to a multiple of 8 bytes
    assert ctypes.sizeof(lbm.lbm_params_t) == 13 * 8 + 8 + 16 * 4
    assert lbm.lbm_params_t.lattice.offset == 13 * 8 + 8 + 14 * 4
    assert lbm.lbm_params_t.plan_blocks.offset == 13 * 8 + 8 + 15 * 4
    assert ctypes.sizeof(lbm.lbm_stats_t) == 13 * 8 + 6 * 8 + 6 * 4


def test_version_and_strerror(lib):
    assert b"sm_103a" in lib.lbm_version()
    for code in (0, -1, -2, -3, -4, -5, 12345):
        assert lib.lbm_strerror(code)


@pytest.mark.parametrize("bad", [
    dict(tau=0.5), dict(tau=0.4), dict(width=0), dict(height=2), dict(width=40000),
    dict(rho_cell=0.0), dict(growth_rate=-1.0), dict(sigma=-0.1), dict(growth_mode=7),
    dict(front_kind=9), dict(wall_mode=3), dict(negfix_mode=2), dict(y_periodic=2),
    dict(growth_mode="density", rho0=0.0), dict(growth_mode="band", band_rows=0),
    dict(front_kind="sinusoidal", front_kmin=5, front_kmax=2),
])
def test_validate_rejects(bad):
    p = wl.lattice_small()
    p.update(bad)
    assert lbm.lbm_validate(p) == -1


def test_validate_accepts_workloads():
    for fn in wl.WORKLOADS.values():
        assert lbm.lbm_validate(fn()) == 0
        assert lbm.lbm_validate(fn(), "fp64") == 0
    assert lbm.lbm_validate(wl.lattice_small(width=1)) == 0


def test_footprint_scales_with_lattice_and_precision():
    a = lbm.lbm_footprint(wl.lattice_small())
    b = lbm.lbm_footprint(wl.lattice_small(), "fp64")
    c = lbm.lbm_footprint(wl.lattice_edge())
    # two FP32 copies of 9 populations at 4096 x 2048 dominate
    assert c >= 2 * 9 * 4096 * 2048 * 4
    assert b > a
    # rows are padded to 32 columns: width 33 stores as many populations as width 64
    assert lbm.lbm_footprint(wl.lattice_small(width=33)) <= lbm.lbm_footprint(wl.lattice_small(width=64))
    assert lbm.lbm_footprint(wl.lattice_small(width=33)) > lbm.lbm_footprint(wl.lattice_small(width=32))


def test_footprint_rejects_null(lib):
    p = lbm.make_params(wl.lattice_small())
    assert lib.lbm_footprint(ctypes.byref(p), None) == -1
    assert lib.lbm_validate(None) == -1


def test_handle_calls_reject_null(lib):
    assert lib.lbm_step(None, 1) == -1
    assert lib.lbm_stats(None, None) == -1
    assert lib.lbm_front_heights(None, None, None, None) == -1
    lib.lbm_destroy(None)


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    p = lbm.make_params(wl.lattice_small())
    h = ctypes.c_void_p()
    rc = lib.lbm_create(ctypes.byref(p), None, None, 0, ctypes.byref(h))
    assert rc in (-3, -5) and not h.value


def test_eq6_host_helper_matches_mean_and_population_std(lib):
    rng = np.random.default_rng(5)
    for W in (1, 7, 4096):
        h = rng.integers(0, 3000, W).astype(np.int64)
        hbar, w = lbm.lbm_eq6(int(h.sum()), int((h * h).sum()), W)
        assert hbar == h.sum() / W
        assert abs(w - h.std()) <= 1e-12 * max(1.0, h.std())
    assert lib.lbm_eq6(1, 1, 0, None, None) == -1


def test_eq6_n_matches_eq6_pair_by_pair(lib):
    rng = np.random.default_rng(6)
    for W in (1, 37, 4096):
        h = rng.integers(0, 3000, (50, W)).astype(np.int64)
        sums = np.stack([h.sum(1), (h * h).sum(1)], axis=1)
        hbar, w = lbm.lbm_eq6_n(sums, W)
        for k in range(len(sums)):
            assert (hbar[k], w[k]) == lbm.lbm_eq6(int(sums[k, 0]), int(sums[k, 1]), W)
    assert lib.lbm_eq6_n(None, 0, 5, None, None) == 0
    assert lib.lbm_eq6_n(None, 1, 5, None, None) == -1
    assert lib.lbm_eq6_n(None, -1, 5, None, None) == -1
    assert lib.lbm_eq6_n(None, 0, 0, None, None) == -1


def test_plan_capacity_grows_with_growth_rate_and_lattice():
    a = lbm.lbm_plan_capacity(wl.lattice_small())
    b = lbm.lbm_plan_capacity(wl.lattice_small(growth_rate=1e-3))
    c = lbm.lbm_plan_capacity(wl.lattice_edge())
    assert 1024 <= a < b < c
    # no growth: the floor of 1024
    assert lbm.lbm_plan_capacity(wl.lattice_small(growth_mode="none")) == 1024


def test_async_calls_reject_null(lib):
    assert lib.lbm_front_heights_async(None, None, None) == -1
    assert lib.lbm_batch_fused(None) == -1


def test_update_kernel_choices_validate():
    p = wl.lattice_small()
    assert lbm.lbm_validate(p, "fp32") == 0
    for uk, ok64 in (("auto", True), ("plain", True), ("tma", False), ("tma1", False), ("shared", True),
                     ("tma_st", False)):
        q = lbm.make_params(p, "fp64", uk)
        assert (lbm.load_library().lbm_validate(ctypes.byref(q)) == 0) == ok64, uk
        q = lbm.make_params(p, "fp32", uk)
        assert lbm.load_library().lbm_validate(ctypes.byref(q)) == 0, uk
    # the bulk-store form is FP32 only
    assert lbm.load_library().lbm_validate(ctypes.byref(lbm.make_params(p, "fp16", "tma_st"))) == -1
    q = lbm.make_params(p, "fp32", 7)
    assert lbm.load_library().lbm_validate(ctypes.byref(q)) == -1
    # the staged kernels need walls in y
    q = lbm.make_params(dict(p, y_periodic=1), "fp32", "tma")
    assert lbm.load_library().lbm_validate(ctypes.byref(q)) == -1


def test_d2q7_update_kinds_validate():
    """D2Q7 takes the plain-load kernel and its one TMA-staged form (FP32,
    walls in y): kinds auto, plain, tma and shared; not the four-row form or
    the global-injection selector, not 16-bit storage, not tma when periodic
    in y, and no odd H when periodic."""
    p = dict(wl.lattice_small(), lattice="d2q7")
    lib = lbm.load_library()
    for uk, ok in (("auto", True), ("plain", True), ("tma", True), ("shared", True), ("tma1", False),
                   ("tma_sel", False), ("tma_st", False)):
        q = lbm.make_params(p, "fp32", uk)
        assert (lib.lbm_validate(ctypes.byref(q)) == 0) == ok, uk
    for uk, ok in (("auto", True), ("plain", True), ("tma", False), ("shared", True)):
        q = lbm.make_params(p, "fp64", uk)
        assert (lib.lbm_validate(ctypes.byref(q)) == 0) == ok, uk
    assert lbm.lbm_validate(p, "fp16") == -1 and lbm.lbm_validate(p, "bf16") == -1
    per = dict(p, y_periodic=1, front_kind="full", height=64)
    assert lib.lbm_validate(ctypes.byref(lbm.make_params(per, "fp32", "tma"))) == -1
    assert lib.lbm_validate(ctypes.byref(lbm.make_params(per, "fp32", "auto"))) == 0
    assert lbm.lbm_validate(dict(per, height=63)) == -1

"""The C-ABI library builds for sm_103a, loads, and exports every function
that include/rgdbek.h declares (CPU only: no compute calls)."""
import ctypes
import os
import re

import numpy as np

import gpu_util

HEADER = os.path.join(gpu_util.ROOT, "include", "rgdbek.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rgdbek_\w+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    path = gpu_util.build_library()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    gpu_util.build_library()
    import paper_2509_19267_gb300 as rg
    bound = {name for name, _, _ in rg.SIGNATURES}
    assert bound == set(declared_functions())
    for name in bound:
        assert callable(getattr(rg, name, None)) or name in ("rgdbek_default_options",
                                                              "rgdbek_status_string")


def test_host_only_calls():
    gpu_util.build_library()
    import paper_2509_19267_gb300 as rg
    o = rg.default_options()
    assert o.eta_col == 0.5 and o.inner_max == 200 and o.stop_rule == rg.STOP_AUTO
    assert rg.status_string(rg.ERR_BAD_CSR) == "malformed CSR matrix"
    # argument checks happen before any device call
    h = ctypes.c_void_p()
    assert rg._lib.rgdbek_create(ctypes.byref(h), 0, 5, 0, None, None, None, 0, None, None) \
        == rg.ERR_INVALID_ARG
    assert rg._lib.rgdbek_solve(None, None, None, 1e-8, 10, 0, None) == rg.ERR_INVALID_ARG
    assert rg._lib.rgdbek_backward(None, None, None, None, None, None, 1e-8, 10, 0, 0,
                                   None) == rg.ERR_INVALID_ARG
    assert rg._lib.rgdbek_tune_eta(None, None, None, None, 0, 5, 0, None, None) \
        == rg.ERR_INVALID_ARG
    assert rg._lib.rgdbek_tune_teams(None, None, None, 5, 0, None, None) == rg.ERR_INVALID_ARG
    # an unknown precision is rejected by the option check, before the device
    rp = np.array([0, 1], dtype=np.int64)
    ci = np.array([0], dtype=np.int32)
    av = np.array([1.0])
    bad = rg.default_options(precision=2)
    assert rg._lib.rgdbek_create(ctypes.byref(h), 1, 1, 1, rp.ctypes.data, ci.ctypes.data,
                                 av.ctypes.data, 0, ctypes.byref(bad), None) \
        == rg.ERR_INVALID_ARG
    assert rg.default_options().precision == rg.PRECISION_FP64
    # the adaptive inner tolerance factor must be a finite c >= 0 (default 0: off)
    assert rg.default_options().inner_adapt == 0.0
    for c in (-0.5, float("nan")):
        bad = rg.default_options(inner_adapt=c)
        assert rg._lib.rgdbek_create(ctypes.byref(h), 1, 1, 1, rp.ctypes.data, ci.ctypes.data,
                                     av.ctypes.data, 0, ctypes.byref(bad), None) \
            == rg.ERR_INVALID_ARG
    # the column team of the two-team schedule: -1 (one team), 0 (automatic)
    # or a CTA count up to the largest grid
    assert rg.default_options().col_team == 0
    for c in (-2, 1025):
        bad = rg.default_options(col_team=c)
        assert rg._lib.rgdbek_create(ctypes.byref(h), 1, 1, 1, rp.ctypes.data, ci.ctypes.data,
                                     av.ctypes.data, 0, ctypes.byref(bad), None) \
            == rg.ERR_INVALID_ARG


def test_size_limits_rejected_before_any_device_call():
    gpu_util.build_library()
    import numpy as np
    import paper_2509_19267_gb300 as rg
    h = ctypes.c_void_p()
    rp = np.zeros(2, dtype=np.int64)
    for m, n in ((2**31, 5), (5, 2**31), (-1, 5)):
        assert rg._lib.rgdbek_create(ctypes.byref(h), m, n, 0, rp.ctypes.data, None, None, 0,
                                     None, None) == rg.ERR_INVALID_ARG
    bad = rg.default_options(eta_col=1.5)
    assert rg._lib.rgdbek_create(ctypes.byref(h), 1, 1, 0, rp.ctypes.data, None, None, 0,
                                 ctypes.byref(bad), None) == rg.ERR_INVALID_ARG


def test_sampler_draw_bound_rejected_before_any_device_call():
    """s above RGDBEK_MAX_DRAWS_PER_ENTRY (16) draws per weight, or a length
    beyond the static scratch, is refused by the argument checks, which run
    before the allocation-free sampler touches the device (fake non-null
    pointers are never dereferenced on this path)."""
    gpu_util.build_library()
    import paper_2509_19267_gb300 as rg
    fake = ctypes.c_void_p(0x1000)
    lib = rg._lib
    assert lib.rgdbek_sample_noalloc(fake, 1000, 16 * 1000 + 1, 0, 0, 0, 0, fake, fake,
                                     None) == rg.ERR_INVALID_ARG
    assert lib.rgdbek_sample_noalloc(fake, 1000, 2**62, 0, 0, 0, 0, fake, fake,
                                     None) == rg.ERR_INVALID_ARG
    assert lib.rgdbek_sample_noalloc(fake, 262145, 10, 0, 0, 0, 0, fake, fake,
                                     None) == rg.ERR_INVALID_ARG
    assert lib.rgdbek_sample_noalloc(fake, 1000, -1, 0, 0, 0, 0, fake, fake,
                                     None) == rg.ERR_INVALID_ARG
    # rgdbek_sample checks the same bound after its handle check
    assert lib.rgdbek_sample(None, fake, 1000, 16001, 0, 0, 0, 0, fake, None) \
        == rg.ERR_INVALID_ARG

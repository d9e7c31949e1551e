"""The C-ABI library loads without a GPU, exports every symbol include/ufvc.h declares, and its host-built
tables equal the oracle's independently built ones byte for byte (CPU only, no compute on a device)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import oracle
from paper_2606_04410_b300 import build
from paper_2606_04410_b300 import ufvc as U

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "ufvc.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(ufvc_[a-z0-9_]+)\s*\(", txt)))


def test_build_is_current():
    assert os.path.exists(build.build())


def test_exports_every_declared_symbol():
    names = declared_symbols()
    assert len(names) >= 20
    for n in names:
        assert hasattr(U.lib, n), n
    assert set(U.EXPORTS) <= set(names)


def test_tables_byte_equal_to_oracle():
    freq = np.empty((64, 511), np.uint32)
    cum = np.empty((64, 512), np.uint32)
    for qp in (0, 27, 32, 40, 63):
        thr = np.empty(63, np.float32)
        assert U.lib.ufvc_get_tables(None, U._ptr(freq), U._ptr(cum), qp, U._ptr(thr)) == 0
        np.testing.assert_array_equal(thr, oracle.thresholds(qp))
    of, oc = oracle.build_tables()
    np.testing.assert_array_equal(freq, of)
    np.testing.assert_array_equal(cum, oc)


def test_architecture_tables_agree_with_oracle():
    for arch in (0, 1):
        for N in (1, 2, 8):
            assert U.weight_count(arch, N) == oracle.weight_count(arch, N)
        for (H, W) in [(64, 64), (1080, 1920), (480, 854), (2160, 3840), (50, 70)]:
            assert U.latent_dims(arch, W, H) == oracle.latent_dims(arch, H, W)
    co, k, ci = C.c_int(), C.c_int(), C.c_int()
    assert U.lib.ufvc_layer_shape(1, 8, 11 + 8 * 7 + 7, C.byref(co), C.byref(k), C.byref(ci)) == 0
    assert (co.value, k.value, ci.value) == (12, 3, 64)
    assert U.lib.ufvc_layer_shape(1, 8, 11 + 8 * 8, C.byref(co), C.byref(k), C.byref(ci)) == U.UFVC_ERR_ARG


def test_create_rejects_bad_arguments_on_host():
    w = np.zeros(U.weight_count(0, 2), np.float32)
    h = C.c_void_p()
    for cfg in [U.ufvc_config(5, 2, 32, 0, 0), U.ufvc_config(0, 0, 32, 0, 0), U.ufvc_config(0, 2, 0, 0, 0),
                U.ufvc_config(0, 2, 70000, 0, 0), U.ufvc_config(0, 2, 32, 9, 0)]:
        assert U.lib.ufvc_create(C.byref(cfg), U._ptr(w), w.size, C.byref(h)) == U.UFVC_ERR_ARG
    cfg = U.ufvc_config(0, 2, 32, 0, 0)
    assert U.lib.ufvc_create(C.byref(cfg), U._ptr(w), w.size - 1, C.byref(h)) == U.UFVC_ERR_ARG

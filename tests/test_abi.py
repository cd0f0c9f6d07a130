"""CPU checks of the C-ABI library: it loads, exports every entry point that
include/nlc.h declares, and its host-only calls behave (no GPU needed)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2201_05213_gb300 import build as B
from paper_2201_05213_gb300 import nlc as N
from paper_2201_05213_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return N.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "nlc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nlc_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_binding_names():
    assert _declared() == sorted(N.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_abi_version(lib):
    assert N.nlc_abi_version() == 1


@pytest.mark.parametrize("cfg", [(3, 32, 2, 10), (3, 64, 2, 10), (1, 64, 2, 10), (2, 16, 0, 3),
                                 (3, 48, 4, 16)])
def test_num_weights_matches_layout(lib, cfg):
    assert N.nlc_num_weights(*cfg) == synth.num_weights(*cfg)
    # the 3,64,2,10 model of the wavefront configurations has 27,812 parameters
    if cfg == (3, 64, 2, 10):
        assert N.nlc_num_weights(*cfg) == 27812


@pytest.mark.parametrize("bad", [(0, 32, 2, 10), (4, 32, 2, 10), (3, 40, 2, 10), (3, 32, 5, 10),
                                 (3, 32, 2, 0), (3, 32, 2, 17)])
def test_invalid_configs_rejected(lib, bad):
    assert N.nlc_num_weights(*bad) == 0
    with pytest.raises(N.NLCError) as e:
        N.nlc_create(*bad, N.NLC_FP32, np.zeros(10, np.float32))
    assert e.value.code == N.NLC_ERR_UNSUPPORTED


def test_weight_count_mismatch_rejected(lib):
    with pytest.raises(N.NLCError) as e:
        N.nlc_create(3, 32, 2, 10, N.NLC_FP32, np.zeros(5, np.float32))
    assert e.value.code == N.NLC_ERR_ARG


def test_compress_bound(lib):
    # 32 header + 8 per stream + 6 per pixel, rounded to 16
    b = N.nlc_compress_bound([(32, 32)], 0, 1)
    assert b == (32 + 8 * 32 + 6 * 1024 + 15) // 16 * 16
    b = N.nlc_compress_bound([(32, 32)], 0, 0)
    assert b == (32 + 8 + 6 * 1024 + 15) // 16 * 16
    # patches: 2048x2048 in 256 patches has 8 x 2048 row streams
    b = N.nlc_compress_bound([(2048, 2048)], 256, 1)
    assert b == (32 + 8 * 8 * 2048 + 6 * 2048 * 2048 + 15) // 16 * 16
    assert N.nlc_compress_bound([(0, 5), (7, 0)], 0, 1) == 32 + 32
    with pytest.raises(N.NLCError):
        N.nlc_compress_bound([(-1, 5)], 0, 1)


def test_null_arguments_rejected(lib):
    assert lib.nlc_destroy(None) == N.NLC_OK
    assert lib.nlc_sync_status(None, None) == N.NLC_ERR_ARG
    assert lib.nlc_compress(None, None, 0, 0, 1, None, 0, None, None) == N.NLC_ERR_ARG
    assert lib.nlc_decompress(None, None, None, None, 0, 0, 1, 1, None) == N.NLC_ERR_ARG
    assert b"bad arguments" in lib.nlc_last_error()

"""Host-side argument handling of the Python binding (no GPU, no library calls)."""
import numpy as np
import pytest

from paper_2211_07983_gb300 import api, _lib


class _FakeState:
    def __init__(self, n_inst):
        self.n_inst = n_inst


def test_precision_names_map_to_the_abi_values():
    assert api._precision("fp64") == _lib.PRECISION_FP64 == 0
    assert api._precision("mixed") == _lib.PRECISION_MIXED == 1
    with pytest.raises(ValueError):
        api._precision("fp32")


def test_theta_shapes_for_single_and_batched_states():
    assert api._n_theta(_FakeState(1), np.zeros(7)) == 7
    assert api._n_theta(_FakeState(3), np.zeros((3, 7))) == 7
    with pytest.raises(ValueError):
        api._n_theta(_FakeState(3), np.zeros(7))          # a batch needs one row per instance
    with pytest.raises(ValueError):
        api._n_theta(_FakeState(3), np.zeros((2, 7)))


def test_config_struct_matches_the_header_layout():
    import ctypes
    # int32 max_bond, double cutoff, int32 precision, int32 checkpoint_every, void* stream
    assert ctypes.sizeof(_lib.MpsConfig) == 32
    assert _lib.MpsConfig.cutoff.offset == 8 and _lib.MpsConfig.cuda_stream.offset == 24

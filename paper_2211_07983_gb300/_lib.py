"""ctypes binding of libmps (include/mps.h): argument marshalling only.

Loading fails loudly if libmps.so has not been built; there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmps.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "mps.h")

c_int32, c_int64, c_double, c_void_p = ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p
c_uint64, c_uint8 = ctypes.c_uint64, ctypes.c_uint8
P = ctypes.POINTER

STATUS = {0: "MPS_OK", 1: "MPS_EINVAL", 2: "MPS_ENOMEM", 3: "MPS_ECUDA", 4: "MPS_ENOCONV", 5: "MPS_ENUMERIC",
          6: "MPS_ETIMEOUT"}
PRECISION_FP64 = 0
PRECISION_MIXED = 1


class MpsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class MpsConfig(ctypes.Structure):
    _fields_ = [("max_bond", c_int32), ("cutoff", c_double), ("precision", c_int32),
                ("checkpoint_every", c_int32), ("cuda_stream", c_void_p)]


class MpsGate(ctypes.Structure):
    _fields_ = [("bond", c_int32), ("theta_idx", c_int32), ("rz_site", c_int32), ("pad_", c_int32),
                ("theta_scale", c_double), ("mat", c_double * 32), ("pre", c_double * 32),
                ("post", c_double * 32)]


class MpsHamiltonian(ctypes.Structure):
    _fields_ = [("n_terms", c_int32), ("x_mask", P(c_uint64)), ("z_mask", P(c_uint64)), ("coeff", P(c_double))]


# numpy view of mps_gate (same layout as the C struct)
GATE_DTYPE = np.dtype([("bond", "<i4"), ("theta_idx", "<i4"), ("rz_site", "<i4"), ("pad_", "<i4"),
                       ("theta_scale", "<f8"), ("mat", "<f8", (32,)), ("pre", "<f8", (32,)),
                       ("post", "<f8", (32,))])
assert GATE_DTYPE.itemsize == ctypes.sizeof(MpsGate)

_SIGS = {
    "mps_build_hamiltonian": (c_int32, [c_int32, P(c_double), P(c_double), c_int64, P(c_uint64), P(c_uint64),
                                        P(c_double), P(c_int64)]),
    "mps_compile_excitations": (c_int32, [c_int32, P(c_int32), c_int32, c_int64, c_void_p, P(c_int64)]),
    "mps_init_product": (c_int32, [c_int32, P(c_uint8), P(MpsConfig), P(c_void_p)]),
    "mps_init_product_batch": (c_int32, [c_int32, c_int32, P(c_uint8), P(MpsConfig), P(c_void_p)]),
    "mps_state_instances": (c_int32, [c_void_p, P(c_int32)]),
    "mps_read_state_instance": (c_int32, [c_void_p, c_int32, P(c_int32), P(c_double), P(c_double)]),
    "mps_clone": (c_int32, [c_void_p, P(c_void_p)]),
    "mps_read_state": (c_int32, [c_void_p, P(c_int32), P(c_double), P(c_double)]),
    "mps_circuit_create": (c_int32, [c_int32, c_void_p, c_int32, P(c_void_p)]),
    "mps_circuit_free": (None, [c_void_p]),
    "mps_hamiltonian_create": (c_int32, [c_int32, P(MpsHamiltonian), P(c_void_p)]),
    "mps_hamiltonian_free": (None, [c_void_p]),
    "mps_apply_circuit": (c_int32, [c_void_p, c_void_p, c_int32, c_void_p, c_int32]),
    "mps_apply_circuit_dev": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32]),
    "mps_energy": (c_int32, [c_void_p, P(MpsHamiltonian), c_void_p]),
    "mps_energy_dev": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "mps_energy_cotangent_dev": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p]),
    "mps_energy_grad": (c_int32, [c_void_p, c_void_p, c_int32, c_void_p, c_int32, P(MpsHamiltonian), c_void_p,
                                  c_void_p, c_void_p]),
    "mps_energy_grad_dev": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_void_p, c_void_p, c_void_p,
                                      c_void_p]),
    "mps_set_svd_policy": (c_int32, [c_void_p, c_int32]),
    "mps_svd_tune": (c_int32, [c_int32, c_int32, c_void_p, c_int32, c_int32, c_int32, c_void_p]),
    "mps_set_svd_tiles": (c_int32, [c_int32, c_void_p]),
    "mps_energy_grad_multi": (c_int32, [c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                        c_void_p]),
    "mps_svd_dev": (c_int32, [c_int32, c_int32, c_void_p, c_int32, c_double, c_void_p, c_void_p, c_void_p,
                              c_void_p]),
    "mps_zgemm_mixed_dev": (c_int32, [c_int32, c_int32, c_int32, c_void_p, c_int32, c_int32, c_void_p, c_int32,
                                      c_int32, c_void_p, c_int32, c_int32]),
    "mps_energy_grad_shard_begin": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_void_p, c_void_p,
                                              c_void_p]),
    "mps_energy_grad_shard_end": (c_int32, [c_void_p, c_void_p, c_int32, c_void_p, c_void_p, c_void_p]),
    "mps_cotangent_size": (c_int32, [c_void_p, P(c_int64)]),
    "mps_profile": (c_int32, [c_void_p, c_int32]),
    "mps_profile_read": (c_int32, [c_void_p, c_void_p]),
    "mps_profile_svd_phases": (c_int32, [c_void_p, c_void_p]),
    "mps_free": (None, [c_void_p]),
    "mps_last_error": (ctypes.c_char_p, []),
    "mps_kernel_launches": (c_int64, []),
}

_lib = None


def header_symbols() -> list[str]:
    """Every function the public header declares."""
    with open(HEADER) as f:
        text = f.read()
    return sorted(set(re.findall(r"\b(mps_[a-z_]+)\s*\(", text)) - {"mps_status"})


def load() -> ctypes.CDLL:
    """Load libmps.so (raises if it is missing: the product has no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing; build it with paper_2211_07983_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def check(code: int) -> None:
    if code != 0:
        msg = load().mps_last_error()
        raise MpsError(code, msg.decode() if msg else "")

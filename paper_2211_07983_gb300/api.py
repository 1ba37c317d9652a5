"""Python face of libmps: the same calls as include/mps.h, with numpy / torch arrays.

Every step of the computation runs in libmps; this module only turns Python objects
into pointers and sizes.  Array arguments may be numpy arrays (host) or torch tensors
(host or CUDA); CUDA tensors are passed as device pointers.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import GATE_DTYPE, MpsConfig, MpsHamiltonian, check

P = ctypes.POINTER


def _ptr(a):
    """Data pointer of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr())
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return ctypes.c_void_p(a.ctypes.data)


def _f64(a):
    if hasattr(a, "data_ptr"):
        import torch
        if a.dtype != torch.float64:
            raise TypeError("float64 tensor expected")
        return a
    return np.ascontiguousarray(a, dtype=np.float64)


def _precision(name: str) -> int:
    if name not in ("fp64", "mixed"):
        raise ValueError('precision must be "fp64" or "mixed"')
    return _lib.PRECISION_FP64 if name == "fp64" else _lib.PRECISION_MIXED


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream      # torch.cuda.Stream


# ---- step S0: host builders ---------------------------------------------------------------

def build_hamiltonian(h: np.ndarray, eri: np.ndarray):
    """mps_build_hamiltonian: integrals -> (x_mask, z_mask, coeff) in canonical order."""
    lib = _lib.load()
    n = int(h.shape[0])
    h = np.ascontiguousarray(h, dtype=np.float64)
    eri = np.ascontiguousarray(eri, dtype=np.float64)
    cnt = ctypes.c_int64(0)
    code = lib.mps_build_hamiltonian(n, h.ctypes.data_as(P(ctypes.c_double)),
                                     eri.ctypes.data_as(P(ctypes.c_double)), 0, None, None, None,
                                     ctypes.byref(cnt))
    if code != 1 or cnt.value <= 0:
        check(code)
    m = cnt.value
    x = np.zeros(m, dtype=np.uint64)
    z = np.zeros(m, dtype=np.uint64)
    c = np.zeros(m, dtype=np.float64)
    check(lib.mps_build_hamiltonian(n, h.ctypes.data_as(P(ctypes.c_double)), eri.ctypes.data_as(P(ctypes.c_double)),
                                    m, x.ctypes.data_as(P(ctypes.c_uint64)), z.ctypes.data_as(P(ctypes.c_uint64)),
                                    c.ctypes.data_as(P(ctypes.c_double)), ctypes.byref(cnt)))
    return x, z, c


def compile_excitations(n: int, excitations) -> np.ndarray:
    """mps_compile_excitations: [(i, j, a, b)] -> structured array of mps_gate (GATE_DTYPE)."""
    lib = _lib.load()
    exc = np.ascontiguousarray(np.asarray(excitations, dtype=np.int32).reshape(-1, 4))
    cnt = ctypes.c_int64(0)
    code = lib.mps_compile_excitations(n, exc.ctypes.data_as(P(ctypes.c_int32)), len(exc), 0, None,
                                       ctypes.byref(cnt))
    if code != 1 or cnt.value < 0:
        check(code)
    gates = np.zeros(cnt.value, dtype=GATE_DTYPE)
    check(lib.mps_compile_excitations(n, exc.ctypes.data_as(P(ctypes.c_int32)), len(exc), cnt.value,
                                      ctypes.c_void_p(gates.ctypes.data), ctypes.byref(cnt)))
    return gates


# ---- handles --------------------------------------------------------------------------------

class State:
    """mps_state: an MPS resident on the GPU (mps_init_product[_batch] / mps_clone / mps_free).

    A state may hold n_inst instances (product_batch); per-call arrays then carry one row per
    instance (theta [n_inst, n_theta], E [n_inst], grad [n_inst, n_theta]).
    """

    def __init__(self, handle, n, n_inst=1):
        self._h = handle
        self.n = n
        self.n_inst = n_inst

    @classmethod
    def product(cls, bits, max_bond: int, cutoff: float, checkpoint_every: int = 0, stream=None,
                precision: str = "fp64"):
        """precision: "fp64", or "mixed" (bond contractions and Pauli sweeps in 3xTF32 on the
        tensor cores; SVD, SVD adjoint and sums in FP64)."""
        lib = _lib.load()
        bits = np.ascontiguousarray(bits, dtype=np.uint8)
        cfg = MpsConfig(max_bond, cutoff, _precision(precision), checkpoint_every, _stream_handle(stream))
        h = ctypes.c_void_p()
        check(lib.mps_init_product(len(bits), bits.ctypes.data_as(P(ctypes.c_uint8)), ctypes.byref(cfg),
                                   ctypes.byref(h)))
        return cls(h, len(bits))

    @classmethod
    def product_batch(cls, bits_rows, max_bond: int, cutoff: float, checkpoint_every: int = 0, stream=None,
                      precision: str = "fp64"):
        """mps_init_product_batch: one product state per row of `bits_rows` ([n_inst, n])."""
        lib = _lib.load()
        bits = np.ascontiguousarray(np.atleast_2d(bits_rows), dtype=np.uint8)
        cfg = MpsConfig(max_bond, cutoff, _precision(precision), checkpoint_every, _stream_handle(stream))
        h = ctypes.c_void_p()
        check(lib.mps_init_product_batch(bits.shape[0], bits.shape[1], bits.ctypes.data_as(P(ctypes.c_uint8)),
                                         ctypes.byref(cfg), ctypes.byref(h)))
        return cls(h, bits.shape[1], bits.shape[0])

    def clone(self):
        h = ctypes.c_void_p()
        check(_lib.load().mps_clone(self._h, ctypes.byref(h)))
        return State(h, self.n, self.n_inst)

    def read(self, inst: int = 0):
        """(dims, lambdas per bond, site tensors) of one instance, copied to the host."""
        lib = _lib.load()
        dims = np.zeros(self.n + 1, dtype=np.int32)
        check(lib.mps_read_state_instance(self._h, inst, dims.ctypes.data_as(P(ctypes.c_int32)), None, None))
        nl = int(dims[1:-1].sum())
        ne = int(sum(dims[s] * 2 * dims[s + 1] for s in range(self.n)))
        lam = np.zeros(max(nl, 1))
        ten = np.zeros(2 * max(ne, 1))
        check(lib.mps_read_state_instance(self._h, inst, dims.ctypes.data_as(P(ctypes.c_int32)),
                                          lam.ctypes.data_as(P(ctypes.c_double)),
                                          ten.ctypes.data_as(P(ctypes.c_double))))
        lams, o = [], 0
        for b in range(1, self.n):
            lams.append(lam[o:o + dims[b]].copy())
            o += dims[b]
        cplx = ten[: 2 * ne].view(np.complex128)
        B, o = [], 0
        for s in range(self.n):
            e = dims[s] * 2 * dims[s + 1]
            B.append(cplx[o:o + e].reshape(dims[s], 2, dims[s + 1]).copy())
            o += e
        return dims, lams, B

    def set_svd_policy(self, one_cta: bool) -> None:
        """mps_set_svd_policy: True = one CTA per gate SVD always (for many concurrent problems),
        False = automatic (the cooperative whole-GPU SVD for matrices above 128 on a side)."""
        check(_lib.load().mps_set_svd_policy(self._h, 1 if one_cta else 0))

    def profile(self, enable: bool = True) -> None:
        """mps_profile: time every gate SVD with CUDA events and count its flops."""
        check(_lib.load().mps_profile(self._h, 1 if enable else 0))

    def profile_read(self) -> dict:
        """mps_profile_read: SVD time (ms), launches, FP64 and FP32 flops since the last read."""
        out = np.zeros(6)
        check(_lib.load().mps_profile_read(self._h, _ptr(out)))
        return {"svd_ms": float(out[0]), "svd_launches": int(out[1]), "fp64_flops": float(out[2]),
                "fp32_flops": float(out[3]), "svd_ms_device": float(out[4]), "svd_launches_device": int(out[5])}

    def profile_phases(self) -> dict:
        """mps_profile_svd_phases: SVD time per phase (ms) and sweeps, gathered by profile_read."""
        out = np.zeros(6)
        check(_lib.load().mps_profile_svd_phases(self._h, _ptr(out)))
        return {"fp32_sweeps_ms": float(out[0]), "reform_ms": float(out[1]), "fp64_sweeps_ms": float(out[2]),
                "output_ms": float(out[3]), "fp32_sweeps": float(out[4]), "fp64_sweeps": float(out[5])}

    def free(self):
        if self._h is not None and self._h.value:
            _lib.load().mps_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Circuit:
    """mps_circuit: a gate list uploaded once."""

    def __init__(self, n: int, gates: np.ndarray):
        gates = np.ascontiguousarray(gates, dtype=GATE_DTYPE)
        self.n, self.n_gates = n, len(gates)
        self.n_theta = int(gates["theta_idx"].max()) + 1 if len(gates) else 0
        h = ctypes.c_void_p()
        check(_lib.load().mps_circuit_create(n, ctypes.c_void_p(gates.ctypes.data), len(gates), ctypes.byref(h)))
        self._h = h

    def __del__(self):
        try:
            if self._h is not None and self._h.value:
                _lib.load().mps_circuit_free(self._h)
        except Exception:
            pass


def _ham_struct(x, z, c):
    x = np.ascontiguousarray(x, dtype=np.uint64)
    z = np.ascontiguousarray(z, dtype=np.uint64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    hs = MpsHamiltonian(len(c), x.ctypes.data_as(P(ctypes.c_uint64)), z.ctypes.data_as(P(ctypes.c_uint64)),
                        c.ctypes.data_as(P(ctypes.c_double)))
    return hs, (x, z, c)


class Hamiltonian:
    """mps_hamiltonian_dev: Pauli strings + sweep trie uploaded once."""

    def __init__(self, n: int, x, z, c):
        hs, keep = _ham_struct(x, z, c)
        h = ctypes.c_void_p()
        check(_lib.load().mps_hamiltonian_create(n, ctypes.byref(hs), ctypes.byref(h)))
        self._h, self.n = h, n
        # expectations are reported for the non-identity strings only
        self.n_terms = int(np.count_nonzero((keep[0] | keep[1]) != 0))

    def __del__(self):
        try:
            if self._h is not None and self._h.value:
                _lib.load().mps_hamiltonian_free(self._h)
        except Exception:
            pass


# ---- steps S1-S9 ----------------------------------------------------------------------------

def _n_theta(state: State, theta) -> int:
    shape = tuple(theta.shape)
    if state.n_inst == 1 and len(shape) == 1:
        return shape[0]
    if len(shape) != 2 or shape[0] != state.n_inst:
        raise ValueError(f"theta must have shape [{state.n_inst}, n_theta] for this state")
    return shape[1]


def apply_circuit(state: State, circuit: Circuit, theta) -> None:
    """mps_apply_circuit_dev: |state> <- U(theta)|state> (theta: [n_theta] or [n_inst, n_theta])."""
    theta = _f64(theta)
    check(_lib.load().mps_apply_circuit_dev(state._h, circuit._h, _ptr(theta), _n_theta(state, theta)))


def energy(state: State, ham: Hamiltonian, expect=False):
    """mps_energy_dev: E (and optionally Re<P_k>/<psi|psi> in canonical order)."""
    ni = state.n_inst
    E = np.zeros(ni)
    ex = np.zeros((ni, ham.n_terms)) if expect else None
    check(_lib.load().mps_energy_dev(state._h, ham._h, _ptr(E), _ptr(ex)))
    if ni == 1:
        return (float(E[0]), ex[0]) if expect else float(E[0])
    return (E, ex) if expect else E


def energy_cotangent(state: State, ham: Hamiltonian):
    """mps_energy_cotangent_dev: E and dE/dB_s* per site (list of [Dl, 2, Dr] arrays)."""
    dims, _, _ = state.read()
    ne = int(sum(dims[s] * 2 * dims[s + 1] for s in range(state.n)))
    E = np.zeros(state.n_inst)
    buf = np.zeros(2 * max(ne, 1))
    check(_lib.load().mps_energy_cotangent_dev(state._h, ham._h, _ptr(E), _ptr(buf)))
    cplx = buf[: 2 * ne].view(np.complex128)
    out, o = [], 0
    for s in range(state.n):
        e = dims[s] * 2 * dims[s + 1]
        out.append(cplx[o:o + e].reshape(dims[s], 2, dims[s + 1]).copy())
        o += e
    return float(E[0]), out


def energy_grad(state0: State, circuit: Circuit, theta, ham: Hamiltonian, out=None, gate_grad=False):
    """mps_energy_grad_dev: E(theta), dE/dtheta (and dE/dphi per gate) of U(theta)|state0>.

    theta: [n_theta], or [n_inst, n_theta] for a batched state (E [n_inst], grad [n_inst, n_theta]).
    `out`: optional (E, grad) arrays/tensors receiving the results (may be CUDA tensors).
    """
    theta = _f64(theta)
    nth = _n_theta(state0, theta)
    ni = state0.n_inst
    if out is None:
        E_out, g_out = np.zeros(ni), np.zeros((ni, nth) if ni > 1 else nth)
    else:
        E_out, g_out = out
    gg = (np.zeros((ni, circuit.n_gates) if ni > 1 else circuit.n_gates)) if gate_grad else None
    check(_lib.load().mps_energy_grad_dev(state0._h, circuit._h, _ptr(theta), nth, ham._h, _ptr(E_out),
                                          _ptr(g_out), _ptr(gg)))
    if out is not None:
        return out
    E = float(E_out[0]) if ni == 1 else E_out
    return (E, g_out, gg) if gate_grad else (E, g_out)


def energy_grad_multi(states, circuits, thetas, hams, outs=None):
    """mps_energy_grad_multi: E and dE/dtheta of independent problems of uneven size, run
    concurrently.  Problem i is energy_grad(states[i], circuits[i], thetas[i], hams[i]).

    Returns (Es, grads): lists with each problem's E (float, or [n_inst] for a batched state) and
    gradient.  `outs`: optional list of (E, grad) arrays/tensors receiving the results.
    """
    n = len(states)
    if not (len(circuits) == len(thetas) == len(hams) == n) or n == 0:
        raise ValueError("states, circuits, thetas and hams must be non-empty lists of one length")
    thetas = [_f64(t) for t in thetas]
    nth = [_n_theta(s, t) for s, t in zip(states, thetas)]
    if outs is None:
        outs = [(np.zeros(s.n_inst), np.zeros((s.n_inst, k) if s.n_inst > 1 else k)) for s, k in zip(states, nth)]
    P = ctypes.c_void_p * n

    def arr(ptrs):
        return P(*[None if q is None else q.value for q in ptrs])

    check(_lib.load().mps_energy_grad_multi(
        n, arr([s._h for s in states]), arr([c._h for c in circuits]), arr([_ptr(t) for t in thetas]),
        (ctypes.c_int32 * n)(*nth), arr([h._h for h in hams]), arr([_ptr(o[0]) for o in outs]),
        arr([_ptr(o[1]) for o in outs])))
    Es = [float(o[0][0]) if s.n_inst == 1 and isinstance(o[0], np.ndarray) else o[0] for s, o in zip(states, outs)]
    return Es, [o[1] for o in outs]


# ---- the host-argument calls of include/mps.h (gate list and Hamiltonian passed per call) -----

def _gates_arg(gates):
    gates = np.ascontiguousarray(gates, dtype=GATE_DTYPE)
    return gates, ctypes.c_void_p(gates.ctypes.data) if len(gates) else None


def apply_circuit_host(state: State, gates, theta) -> None:
    """mps_apply_circuit: gate list as a host array of mps_gate (GATE_DTYPE)."""
    theta = _f64(theta)
    gates, gp = _gates_arg(gates)
    check(_lib.load().mps_apply_circuit(state._h, gp, len(gates), _ptr(theta), _n_theta(state, theta)))


def energy_host(state: State, x, z, c):
    """mps_energy: Hamiltonian as host arrays (x_mask, z_mask, coeff)."""
    hs, _keep = _ham_struct(x, z, c)
    E = np.zeros(state.n_inst)
    check(_lib.load().mps_energy(state._h, ctypes.byref(hs), _ptr(E)))
    return float(E[0]) if state.n_inst == 1 else E


def energy_grad_host(state0: State, gates, theta, x, z, c, gate_grad=False):
    """mps_energy_grad: gate list and Hamiltonian as host arrays."""
    theta = _f64(theta)
    nth = _n_theta(state0, theta)
    gates, gp = _gates_arg(gates)
    hs, _keep = _ham_struct(x, z, c)
    ni = state0.n_inst
    E = np.zeros(ni)
    g = np.zeros((ni, nth) if ni > 1 else nth)
    gg = (np.zeros((ni, len(gates)) if ni > 1 else len(gates))) if gate_grad else None
    check(_lib.load().mps_energy_grad(state0._h, gp, len(gates), _ptr(theta), nth, ctypes.byref(hs), _ptr(E),
                                      _ptr(g), _ptr(gg)))
    Ev = float(E[0]) if ni == 1 else E
    return (Ev, g, gg) if gate_grad else (Ev, g)


def cotangent_size(state: State) -> int:
    """mps_cotangent_size: doubles of the state's cotangent buffer (all instances)."""
    n = ctypes.c_int64(0)
    check(_lib.load().mps_cotangent_size(state._h, ctypes.byref(n)))
    return int(n.value)


def energy_grad_shard_begin(state0: State, circuit: Circuit, theta, ham_shard: Hamiltonian):
    """mps_energy_grad_shard_begin: forward pass, then E_r and the cotangent of this shard's strings.

    Returns (E_r, Bbar_r) as float64 CUDA tensors ([n_inst] and [cotangent_size]) to be summed
    over the ranks before energy_grad_shard_end."""
    import torch
    theta = _f64(theta)
    nth = _n_theta(state0, theta)
    E = torch.zeros(state0.n_inst, dtype=torch.float64, device="cuda")
    Bbar = torch.zeros(cotangent_size(state0), dtype=torch.float64, device="cuda")
    check(_lib.load().mps_energy_grad_shard_begin(state0._h, circuit._h, _ptr(theta), nth, ham_shard._h, _ptr(E),
                                                  _ptr(Bbar)))
    return E, Bbar


def energy_grad_shard_end(state0: State, circuit: Circuit, n_theta: int, Bbar, gate_grad: bool = False):
    """mps_energy_grad_shard_end: the reverse pass from the summed cotangent -> dE/dtheta."""
    ni = state0.n_inst
    g = np.zeros((ni, n_theta) if ni > 1 else n_theta)
    gg = (np.zeros((ni, circuit.n_gates) if ni > 1 else circuit.n_gates)) if gate_grad else None
    check(_lib.load().mps_energy_grad_shard_end(state0._h, circuit._h, n_theta, _ptr(Bbar), _ptr(g), _ptr(gg)))
    return (g, gg) if gate_grad else g


def svd(A: np.ndarray, D: int, eps: float):
    """mps_svd_dev: the GPU gate SVD of one complex matrix -> (s, V, W = A V, k)."""
    A = np.ascontiguousarray(A, dtype=np.complex128)
    m, ncol = A.shape
    K = min(m, ncol)
    s = np.zeros(K)
    V = np.zeros((ncol, K), dtype=np.complex128)
    W = np.zeros((m, K), dtype=np.complex128)
    k = np.zeros(1, dtype=np.int32)
    check(_lib.load().mps_svd_dev(m, ncol, _ptr(A), D, eps, _ptr(s), _ptr(V), _ptr(W), _ptr(k)))
    return s, V, W, int(k[0])


_OPS = {"N": 0, "T": 1, "H": 2, "C": 3}
_ENGINES = {"mma_sync": 0, "tcgen05": 1, "fp64": 2}


def zgemm(A, B, opA: str = "N", opB: str = "N", engine: str = "tcgen05"):
    """mps_zgemm_mixed_dev: C = op(A) op(B) on the GPU with one of the contraction kernels.

    A, B: complex128 CUDA tensors (2-d, row-major); returns C as a complex128 CUDA tensor.
    """
    import torch
    M = A.shape[0] if opA in ("N", "C") else A.shape[1]
    K = A.shape[1] if opA in ("N", "C") else A.shape[0]
    N = B.shape[1] if opB in ("N", "C") else B.shape[0]
    A = A.contiguous()
    B = B.contiguous()
    C = torch.zeros((M, N), dtype=torch.complex128, device=A.device)
    check(_lib.load().mps_zgemm_mixed_dev(M, N, K, ctypes.c_void_p(A.data_ptr()), A.shape[1], _OPS[opA],
                                          ctypes.c_void_p(B.data_ptr()), B.shape[1], _OPS[opB],
                                          ctypes.c_void_p(C.data_ptr()), N, _ENGINES[engine]))
    return C


def kernel_launches() -> int:
    return int(_lib.load().mps_kernel_launches())

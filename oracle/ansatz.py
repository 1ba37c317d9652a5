"""Oracle: UCCSD excitations -> nearest-neighbour two-qubit gate list.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Paper passages followed:
* Sec. 2, Eq. (uccansatz) and the cluster operator T = sum theta^a_i T^a_i +
  1/4 sum theta^{ab}_{ij} T^{ab}_{ij}: one angle per excitation, the 1/4 absorbing
  the four index orderings of a double, so each excitation contributes
  exp(theta (T - T+)).
* Sec. 2, Trotter step: first order (k = 1); the excitations are applied in list
  order, the first one first.  Each exp(theta (T - T+)) is the exact product of
  the rotations of its mutually commuting Jordan-Wigner strings, realised as the
  "V-shaped" block basis change -> CNOT ladder -> Rz -> ladder^-1 -> basis^-1.
* Sec. 3, gate fusion: single-qubit gates are absorbed into two-qubit gates.

Readings (where the paper gives no detail):
* exp(theta (T - T+)) = exp(i theta sum_P c_P P) (T - T+ is anti-Hermitian, its
  Jordan-Wigner coefficients are i*c_P).  exp(i theta c P) = exp(-i phi/2 P) with
  phi = -2 c theta; Rz(phi) = diag(e^{-i phi/2}, e^{+i phi/2}).
* Basis changes: X = H Z H, Y = W^+ Z W with W = Rx(pi/2) = (I - iX)/sqrt 2.
* Ladder over [a, b]: for s = a .. b-1, CNOT(control s, target s+1) when site
  s+1 carries X/Y/Z, SWAP(s, s+1) when it carries I (moves the running parity
  past a site that must not enter it); the parity ends on site b.
* Strings of one excitation are applied in canonical string order
  (oracle.pauli.sort_key), which makes consecutive ladders share their lower part.
* Peephole rules, in this order:
  (1) cancel adjacent inverse pairs (H H, Rx(pi/2) Rx(-pi/2), equal CNOTs, SWAP SWAP)
      when no other gate touches their qubits in between, repeatedly (stack);
  (2) absorb each single-qubit gate into the nearest following two-qubit gate
      touching its qubit, else into the nearest preceding one;
  (3) merge maximal runs of two-qubit gates on the same bond with nothing touching
      either qubit in between, unless both carry an Rz angle.
* Two-qubit gate index order (i_n, i_{n+1}), i_n major; CNOT control = lower site.
"""
from __future__ import annotations

import bisect
from dataclasses import dataclass

import numpy as np

from . import pauli

SQ2 = 1.0 / np.sqrt(2.0)
I2 = np.eye(2, dtype=complex)
I4 = np.eye(4, dtype=complex)
HAD = np.array([[1, 1], [1, -1]], dtype=complex) * SQ2
RXP = np.array([[1, -1j], [-1j, 1]], dtype=complex) * SQ2      # Rx(+pi/2)
RXM = np.array([[1, 1j], [1j, 1]], dtype=complex) * SQ2        # Rx(-pi/2)
CNOT = np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], dtype=complex)
SWAP = np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]], dtype=complex)
ONE_Q = {"H": HAD, "RXP": RXP, "RXM": RXM}
TWO_Q = {"CNOT": CNOT, "SWAP": SWAP, "ID": I4}
INVERSE_1Q = {"H": "H", "RXP": "RXM", "RXM": "RXP"}


def rz(phi: float) -> np.ndarray:
    return np.diag([np.exp(-0.5j * phi), np.exp(0.5j * phi)])


def drz(phi: float) -> np.ndarray:
    return np.diag([-0.5j * np.exp(-0.5j * phi), 0.5j * np.exp(0.5j * phi)])


@dataclass
class Gate:
    """Fused nearest-neighbour gate on sites (bond, bond+1).

    Fixed:      G = mat.
    Parametric: G(phi) = post @ Rz_site(phi) @ pre, phi = scale * theta[theta_idx],
                Rz on the lower site (rz_site = 0) or the upper site (1).
    """
    bond: int
    mat: np.ndarray = None
    theta_idx: int = -1
    scale: float = 0.0
    rz_site: int = 0
    pre: np.ndarray = None
    post: np.ndarray = None

    @property
    def parametric(self) -> bool:
        return self.theta_idx >= 0

    def phi(self, theta) -> float:
        return self.scale * float(theta[self.theta_idx])

    def matrix(self, theta=None, phi=None) -> np.ndarray:
        if not self.parametric:
            return self.mat
        if phi is None:
            phi = self.phi(theta)
        r = np.kron(rz(phi), I2) if self.rz_site == 0 else np.kron(I2, rz(phi))
        return self.post @ r @ self.pre

    def dmatrix(self, theta=None, phi=None) -> np.ndarray:
        """dG/dphi (zero for fixed gates)."""
        if not self.parametric:
            return np.zeros((4, 4), dtype=complex)
        if phi is None:
            phi = self.phi(theta)
        r = np.kron(drz(phi), I2) if self.rz_site == 0 else np.kron(I2, drz(phi))
        return self.post @ r @ self.pre


# ---- excitation generators ---------------------------------------------------

def excitation_strings(exc, n: int):
    """T - T+ = sum_P (i c_P) P  ->  [(x, z, c_P)] in canonical order.

    exc = (i, j, a, b); a single i->a has j = b = -1 and T = a+_a a_i; a double has
    T = a+_a a+_b a_j a_i.
    """
    i, j, a, b = exc
    cre = pauli.jw_creation
    ann = pauli.jw_annihilation
    acc = pauli.ExactAccumulator()
    if j < 0:
        fac, fac_h, w = [cre(a), ann(i)], [cre(i), ann(a)], 0.25
    else:
        fac, fac_h, w = [cre(a), cre(b), ann(j), ann(i)], [cre(i), cre(j), ann(b), ann(a)], 0.0625
    for (k, x, z) in pauli.product_terms(fac):
        acc.add(k, x, z, w)
    for (k, x, z) in pauli.product_terms(fac_h):
        acc.add(k, x, z, -w)
    out = []
    for (x, z), alpha in acc.merged().items():
        if alpha == 0:
            continue
        assert alpha.real == 0.0, "T - T+ must map to purely imaginary coefficients"
        out.append((pauli.sort_key(x, z, n), x, z, alpha.imag))
    out.sort(key=lambda t: t[0])
    strings = [(x, z, c) for (_, x, z, c) in out]
    for s1 in strings:                      # the product formula needs commuting strings
        for s2 in strings:
            e12, _, _ = pauli.mul(s1[0], s1[1], s2[0], s2[1])
            e21, _, _ = pauli.mul(s2[0], s2[1], s1[0], s1[1])
            assert e12 == e21
    return strings


def rotation_primitives(x: int, z: int, theta_idx: int, scale: float):
    """V-shaped block for exp(-i phi/2 P), phi = scale * theta[theta_idx]."""
    a, b = pauli.support_range(x, z)
    sym = {s: pauli.site_symbol(x, z, s) for s in range(a, b + 1)}
    g = []
    for s in range(a, b + 1):
        if sym[s] == "X":
            g.append(("1q", "H", s))
        elif sym[s] == "Y":
            g.append(("1q", "RXP", s))
    ladder = [("2q", "CNOT" if sym[s + 1] != "I" else "SWAP", s) for s in range(a, b)]
    g += ladder
    g.append(("1q", "RZ", b, theta_idx, scale))
    g += ladder[::-1]
    for s in range(a, b + 1):
        if sym[s] == "X":
            g.append(("1q", "H", s))
        elif sym[s] == "Y":
            g.append(("1q", "RXM", s))
    return g


def qubits_of(g):
    return (g[2],) if g[0] == "1q" else (g[2], g[2] + 1)


def is_inverse_pair(h, g) -> bool:
    if h[0] != g[0] or h[2] != g[2]:
        return False
    if g[0] == "1q":
        return g[1] != "RZ" and h[1] != "RZ" and INVERSE_1Q[h[1]] == g[1]
    return h[1] == g[1] and g[1] in ("CNOT", "SWAP")


def cancel_inverse_pairs(prims, n: int):
    """Rule (1): per-qubit stacks; a gate cancels against the gate on top of all its
    qubits' stacks when that gate acts on exactly the same qubits and is its inverse."""
    out = []
    stacks = [[] for _ in range(n)]
    for g in prims:
        qs = qubits_of(g)
        top = stacks[qs[0]][-1] if stacks[qs[0]] else None
        if (top is not None and all(stacks[q] and stacks[q][-1] == top for q in qs)
                and qubits_of(out[top]) == qs and is_inverse_pair(out[top], g)):
            for q in qs:
                stacks[q].pop()
            out[top] = None
            continue
        out.append(g)
        for q in qs:
            stacks[q].append(len(out) - 1)
    return [g for g in out if g is not None]


def one_q_matrix(g, bond):
    w = ONE_Q[g[1]]
    return np.kron(w, I2) if g[2] == bond else np.kron(I2, w)


def absorb_single_qubit(prims, n: int):
    """Rule (2): returns fused two-qubit gates in time order."""
    # a qubit that no two-qubit gate touches gets an identity two-qubit gate at its first use
    touched = set()
    for g in prims:
        if g[0] == "2q":
            touched.update(qubits_of(g))
    fixed = []
    for g in prims:
        if g[0] == "1q" and g[2] not in touched:
            q = g[2]
            fixed.append(("2q", "ID", q if q < n - 1 else q - 1))
            touched.update(qubits_of(fixed[-1]))
        fixed.append(g)
    prims = fixed
    pos = [[] for _ in range(n)]            # positions of two-qubit gates touching each qubit
    for t, g in enumerate(prims):
        if g[0] == "2q":
            for q in qubits_of(g):
                pos[q].append(t)
    before = {t: [] for q in range(n) for t in pos[q]}
    after = {t: [] for t in before}
    for t, g in enumerate(prims):
        if g[0] != "1q":
            continue
        p = pos[g[2]]
        u = bisect.bisect_right(p, t)
        if u < len(p):
            before[p[u]].append(g)
        else:
            after[p[u - 1]].append(g)
    fused = []
    for t, g in enumerate(prims):
        if g[0] != "2q":
            continue
        bond = g[2]
        seq = before[t] + [("core", g[1])] + after[t]
        rz_at = [u for u, e in enumerate(seq) if e[0] == "1q" and e[1] == "RZ"]
        assert len(rz_at) <= 1, "two Rz angles cannot share one fused gate"

        def mat_of(e):
            return TWO_Q[e[1]] if e[0] == "core" else one_q_matrix(e, bond)

        def prod(es):
            m = I4.copy()
            for e in es:                     # time order: later gates multiply from the left
                m = mat_of(e) @ m
            return m

        if not rz_at:
            fused.append(Gate(bond=bond, mat=prod(seq)))
        else:
            r = rz_at[0]
            e = seq[r]
            fused.append(Gate(bond=bond, theta_idx=e[3], scale=e[4],
                              rz_site=0 if e[2] == bond else 1,
                              pre=prod(seq[:r]), post=prod(seq[r + 1:])))
    return fused


def merge_runs(fused, n: int):
    """Rule (3): merge consecutive gates on one bond (at most one Rz angle per gate)."""
    out = []
    last = [None] * n
    for g in fused:
        lo, hi = g.bond, g.bond + 1
        t = last[lo]
        if t is not None and last[hi] == t and out[t].bond == g.bond and not (
                out[t].parametric and g.parametric):
            h = out[t]
            if not h.parametric and not g.parametric:
                h.mat = g.mat @ h.mat
            elif h.parametric:
                h.post = g.mat @ h.post
            else:
                out[t] = Gate(bond=g.bond, theta_idx=g.theta_idx, scale=g.scale,
                              rz_site=g.rz_site, pre=g.pre @ h.mat, post=g.post)
            continue
        out.append(g)
        last[lo] = last[hi] = len(out) - 1
    return out


def primitive_circuit(n: int, excitations):
    prims = []
    for t, exc in enumerate(excitations):
        for (x, z, c) in excitation_strings(exc, n):
            prims += rotation_primitives(x, z, t, -2.0 * c)
    return prims


def compile_circuit(n: int, excitations):
    """Excitations (applied in list order) -> fused nearest-neighbour gates."""
    prims = primitive_circuit(n, excitations)
    prims = cancel_inverse_pairs(prims, n)
    return merge_runs(absorb_single_qubit(prims, n), n)


def circuit_unitary_dense(n: int, gates, theta) -> np.ndarray:
    """Dense 2^n unitary of a fused gate list (small n only)."""
    U = np.eye(2 ** n, dtype=complex)
    for g in gates:
        full = np.kron(np.kron(np.eye(2 ** g.bond), g.matrix(theta)), np.eye(2 ** (n - g.bond - 2)))
        U = full @ U
    return U

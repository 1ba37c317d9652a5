"""Oracle: Pauli strings and the Jordan-Wigner qubit Hamiltonian.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Paper passages followed:
* Sec. 2, Eq. (ham-pbc): H = sum_pq h^p_q a+_p a_q + 1/2 sum_pqrs g^{pq}_{rs} a+_p a+_q a_r a_s.
  Reading: the integrals are given in chemist notation (pq|rs), so the
  two-electron part is 1/2 sum (pq|rs) a+_p a+_r a_s a_q  (g^{pq}_{rs} = (ps|qr)).
* Sec. 2, Eq. (expect-val): after the Jordan-Wigner map, H = sum_k c_k P_k and
  E = sum_k c_k <psi|P_k|psi>.

Representation: an n-qubit Pauli string is a pair of integers (x, z); bit s of
x / z belongs to qubit (site) s.  Per site (x_s, z_s) = (0,0) I, (1,0) X,
(0,1) Z, (1,1) Y, i.e. P(x, z) = tensor_s i^{x_s z_s} X^{x_s} Z^{z_s}.

Jordan-Wigner with |1> = occupied:  a_p = Z_0 ... Z_{p-1} (X_p + i Y_p) / 2.
"""
from __future__ import annotations

import math
from collections import defaultdict

import numpy as np

SYMBOLS = "IXYZ"          # sort order I < X < Y < Z


def popcount(v: int) -> int:
    return bin(v).count("1")


def site_symbol(x: int, z: int, s: int) -> str:
    xb, zb = (x >> s) & 1, (z >> s) & 1
    return {(0, 0): "I", (1, 0): "X", (0, 1): "Z", (1, 1): "Y"}[(xb, zb)]


def to_label(x: int, z: int, n: int) -> str:
    """String label, site 0 first, e.g. 'XZZY'."""
    return "".join(site_symbol(x, z, s) for s in range(n))


def from_label(label: str):
    x = z = 0
    for s, ch in enumerate(label):
        if ch in "XY":
            x |= 1 << s
        if ch in "ZY":
            z |= 1 << s
    return x, z


def mul(x1: int, z1: int, x2: int, z2: int):
    """P(x1,z1) P(x2,z2) = i^e P(x1^x2, z1^z2); returns (e mod 4, x, z).

    Derivation: Z^z1 X^x2 = (-1)^{z1.x2} X^x2 Z^z1 and X^x Z^z = i^{-x.z} P(x,z), so
    e = |x1&z1| + |x2&z2| + 2|z1&x2| - |x3&z3|.  Checked against explicit 2x2
    matrix products in the tests.
    """
    x3, z3 = x1 ^ x2, z1 ^ z2
    e = popcount(x1 & z1) + popcount(x2 & z2) + 2 * popcount(z1 & x2) - popcount(x3 & z3)
    return e % 4, x3, z3


# ---- Jordan-Wigner single-mode operators ------------------------------------
# A "Pauli sum with exact coefficients" is a list of (k, x, z) meaning i^k * 2^-1 * P(x,z)
# per factor; products track the power of i and the power of 1/2 separately.

def jw_annihilation(p: int):
    """a_p = 1/2 Z_<p X_p + i/2 Z_<p Y_p as [(power of i, x, z)], each with weight 1/2."""
    below = (1 << p) - 1
    return [(0, 1 << p, below), (1, 1 << p, below | (1 << p))]


def jw_creation(p: int):
    """a+_p = 1/2 Z_<p X_p - i/2 Z_<p Y_p."""
    below = (1 << p) - 1
    return [(0, 1 << p, below), (3, 1 << p, below | (1 << p))]


def product_terms(factors):
    """Expand a product of single-mode operators into Pauli strings.

    Returns a list of (k, x, z): each term equals i^k * 2^-len(factors) * P(x,z).
    """
    terms = [(0, 0, 0)]
    for f in factors:
        new = []
        for (k, x, z) in terms:
            for (kf, xf, zf) in f:
                e, x3, z3 = mul(x, z, xf, zf)
                new.append(((k + kf + e) % 4, x3, z3))
        terms = new
    return terms


class ExactAccumulator:
    """Collects exact contributions per Pauli string; merges by correctly rounded sums.

    Every contribution is (real number) * i^k with k in 0..3, so it lands exactly in
    the real or the imaginary part.  math.fsum gives the correctly rounded value of
    the exact sum, which makes the merged coefficient independent of the order in
    which contributions arrive.
    """

    def __init__(self):
        self.re = defaultdict(list)
        self.im = defaultdict(list)

    def add(self, k: int, x: int, z: int, value: float):
        if value == 0.0:
            return
        if k == 0:
            self.re[(x, z)].append(value)
        elif k == 2:
            self.re[(x, z)].append(-value)
        elif k == 1:
            self.im[(x, z)].append(value)
        else:
            self.im[(x, z)].append(-value)

    def merged(self):
        keys = set(self.re) | set(self.im)
        return {key: complex(math.fsum(self.re.get(key, [])), math.fsum(self.im.get(key, [])))
                for key in keys}


def accumulate_hamiltonian(h: np.ndarray, eri: np.ndarray) -> ExactAccumulator:
    """All Jordan-Wigner contributions of H (Eq. ham-pbc, chemist-notation reading)."""
    n = h.shape[0]
    acc = ExactAccumulator()
    ann = [jw_annihilation(p) for p in range(n)]
    cre = [jw_creation(p) for p in range(n)]
    for p in range(n):
        for q in range(n):
            v = float(h[p, q])
            if v == 0.0:
                continue
            for (k, x, z) in product_terms([cre[p], ann[q]]):
                acc.add(k, x, z, v * 0.25)
    nz = np.argwhere(eri != 0.0)
    for (p, q, r, s) in nz:
        if p == r or q == s:          # a+_p a+_p = 0 and a_s a_s = 0
            continue
        v = float(eri[p, q, r, s])
        # 1/2 (pq|rs) a+_p a+_r a_s a_q ; four factors carry 2^-4
        for (k, x, z) in product_terms([cre[p], cre[r], ann[s], ann[q]]):
            acc.add(k, x, z, v * 0.5 * 0.0625)
    return acc


def sort_key(x: int, z: int, n: int):
    """Canonical order: first non-identity site a, then the symbols from a on (I<X<Y<Z).

    The identity string comes first (a = -1).
    """
    support = x | z
    if support == 0:
        return (-1, ())
    a = (support & -support).bit_length() - 1
    return (a, tuple(SYMBOLS.index(site_symbol(x, z, s)) for s in range(a, n)))


def support_range(x: int, z: int):
    """(a, b): first and last non-identity site; (-1, -1) for the identity."""
    support = x | z
    if support == 0:
        return (-1, -1)
    return ((support & -support).bit_length() - 1, support.bit_length() - 1)


class PauliHamiltonian:
    """Merged, filtered, canonically ordered weighted Pauli strings + sweep batches."""

    def __init__(self, n, x, z, coeff):
        self.n = n
        self.x = list(x)
        self.z = list(z)
        self.coeff = np.asarray(coeff, dtype=np.float64)
        starts = [support_range(a, b)[0] for a, b in zip(self.x, self.z)]
        # sweep batches: maximal runs of strings sharing the first non-identity site
        self.batch_offsets = [0]
        for t in range(1, len(starts)):
            if starts[t] != starts[t - 1]:
                self.batch_offsets.append(t)
        self.batch_offsets.append(len(starts))

    def __len__(self):
        return len(self.x)

    def labels(self):
        return [to_label(a, b, self.n) for a, b in zip(self.x, self.z)]


def jw_hamiltonian(h: np.ndarray, eri: np.ndarray, drop_rel: float = 1e-14) -> PauliHamiltonian:
    """Integrals -> merged Jordan-Wigner strings in canonical order.

    Strings with |c| <= drop_rel * max|c| are exact cancellations and are dropped.
    The imaginary parts of a Hermitian H cancel exactly; that is asserted.
    """
    n = h.shape[0]
    merged = jw_merge(accumulate_hamiltonian(h, eri))
    cmax = max((abs(c) for c in merged.values()), default=0.0)
    keep = []
    for (x, z), c in merged.items():
        if abs(c) <= drop_rel * cmax:
            continue
        assert abs(c.imag) <= drop_rel * cmax, "non-Hermitian Pauli coefficient"
        keep.append((sort_key(x, z, n), x, z, c.real))
    keep.sort(key=lambda t: t[0])
    return PauliHamiltonian(n, [t[1] for t in keep], [t[2] for t in keep], [t[3] for t in keep])


def jw_merge(acc: ExactAccumulator):
    return acc.merged()


# ---- dense matrices (small n only) -------------------------------------------

_PAULI = {
    "I": np.eye(2, dtype=complex),
    "X": np.array([[0, 1], [1, 0]], dtype=complex),
    "Y": np.array([[0, -1j], [1j, 0]], dtype=complex),
    "Z": np.array([[1, 0], [0, -1]], dtype=complex),
}


def site_matrix(x: int, z: int, s: int) -> np.ndarray:
    return _PAULI[site_symbol(x, z, s)]


def pauli_dense(x: int, z: int, n: int) -> np.ndarray:
    """Dense 2^n matrix; site 0 is the most significant tensor factor."""
    m = np.ones((1, 1), dtype=complex)
    for s in range(n):
        m = np.kron(m, site_matrix(x, z, s))
    return m


def hamiltonian_dense(ham: PauliHamiltonian) -> np.ndarray:
    n = ham.n
    H = np.zeros((2 ** n, 2 ** n), dtype=complex)
    for x, z, c in zip(ham.x, ham.z, ham.coeff):
        H += c * pauli_dense(x, z, n)
    return H

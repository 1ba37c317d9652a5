"""Oracle: MPS circuit simulator, Pauli-string energy and its exact reverse-mode gradient.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Paper passages followed:
* Sec. 3, Eq. (mps): c_{i1..iN} = B^{i1} B^{i2} ... B^{iN}; site tensors B[Dl, 2, Dr].
* Sec. 3, Eq. (hf): product state, D = 1, B^{b_n} = 1, B^{1-b_n} = 0.
* Sec. 3, Eq. (rightcanonicalcondition) and the two-qubit gate update (Hastings'
  technique): C = Q (B_n B_{n+1}); C~ = lambda_{n-1} C; SVD(C~) = U lambda~ V;
  truncate; B~_n = C V^+, B~_{n+1} = V; lambda_n <- lambda~.
* Sec. 3, Eq. (paulistringexp): <Psi|P|Psi> by contracting the 1-D network.
* Sec. 2, Eq. (expect-val): E = sum_k c_k <psi|P_k|psi>.
* Sec. 4, Eqs. (expecgrad), (circuitevolvegrad) and App. A, Eqs. (bp3), (bp4):
  complex reverse-mode rules; the cotangent of a complex X is Xbar = dE/dX*, with
  dE = 2 Re <Xbar, dX>, and a real input theta gets thetabar = 2 Re <Gbar, dG/dtheta>.

Readings:
* Truncation: k = max(1, min(D, #{i : s_i / ||s||_2 > eps})); lambda~ = s_1..k
  renormalised to unit 2-norm; site tensors are not rescaled.
* E is normalised: E = sum_k c_k Re <psi|P_k|psi> / <psi|psi> with full
  contractions (no use of lambda in the energy).
* The gradient is the exact derivative of this truncated forward pass with the
  kept count k held fixed (the "local" approach of Sec. 4 made exact): the SVD is
  differentiated through M = C~^+ C~ = V diag(s^2) V^+ with the full spectrum,
  F_ij = 1/(w_j - w_i), set to 0 for pairs degenerate to within 1e-10 relative (DEGEN_REL)
  or closer than 1e-13 s_1 (DEGEN_ABS);
  singular values at or below 1e-13 s_1 count as exact zeros (NULL_REL).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import pauli

# Pairs of squared singular values with |w_i - w_j| <= DEGEN_REL * max(w_i, w_j) count as
# exactly degenerate: their F_ij is 0.  A rotation inside an exactly degenerate block leaves
# E unchanged, and a singular-value split at rounding level must not be divided by.
DEGEN_REL = 1e-10
# A computed singular value is known to an absolute accuracy of a few ulps of s_1, so two values
# closer than DEGEN_ABS * s_1 are indistinguishable from an exactly degenerate pair as well; for
# values far below s_1 this absolute rule is the one that applies (a degenerate pair at 5e-11 s_1
# comes out split by ~1e-16 s_1, i.e. 2e-6 relative, which the relative rule alone would divide by).
DEGEN_ABS = 1e-13
# Singular values at or below NULL_REL * s_1 are rounding noise of an exactly rank-deficient
# matrix (particle-number and spin symmetry make many two-site tensors rank deficient); the
# adjoint treats them as exact zeros: w_i = 0 and the column (C~ V)_i = 0.
NULL_REL = 1e-13


@dataclass
class MPS:
    B: list                   # site tensors [Dl, 2, Dr], complex128
    lam: list                 # Schmidt vectors of bonds 0..n-2 (float64)

    @property
    def n(self):
        return len(self.B)

    def copy(self):
        return MPS([b.copy() for b in self.B], [l.copy() for l in self.lam])

    def bond_dims(self):
        return [b.shape[2] for b in self.B[:-1]]


def init_product(bits) -> MPS:
    """Eq. (hf): B^{b_n}_{00} = 1, B^{1-b_n}_{00} = 0; all lambda = [1]."""
    B = []
    for b in bits:
        t = np.zeros((1, 2, 1), dtype=complex)
        t[0, int(b), 0] = 1.0
        B.append(t)
    return MPS(B, [np.ones(1) for _ in range(len(bits) - 1)])


def truncation_rank(s: np.ndarray, D: int, eps: float) -> int:
    """k = max(1, min(D, #{i : s_i/||s||_2 > eps and s_i > NULL_REL s_1})).

    Values at rounding level (s_i <= NULL_REL s_1) are numerical zeros and are never kept,
    whatever eps is (only matters for eps < 1e-13).
    """
    norm = math.sqrt(float(np.sum(s * s)))
    if norm == 0.0:
        return 1
    count = int(np.sum((s / norm > eps) & (s > NULL_REL * s[0])))
    return max(1, min(D, count))


def apply_gate(mps: MPS, bond: int, G: np.ndarray, D: int, eps: float, keep_tape=False):
    """Two-qubit gate on sites (bond, bond+1), Sec. 3; returns the tape if asked."""
    n0 = bond
    Bl, Br = mps.B[n0], mps.B[n0 + 1]
    Dl, Dr = Bl.shape[0], Br.shape[2]
    theta4 = two_site(Bl, Br)
    C = np.einsum("xy,ayc->axc", G, theta4.reshape(Dl, 4, Dr)).reshape(Dl, 2, 2, Dr)
    lam_left = mps.lam[n0 - 1] if n0 > 0 else np.ones(1)
    Ct = lam_left[:, None, None, None] * C
    Cm = Ct.reshape(2 * Dl, 2 * Dr)
    U, s, Vh = np.linalg.svd(Cm, full_matrices=True)
    V = Vh.conj().T
    k = truncation_rank(s, D, eps)
    sk = s[:k]
    lam_new = sk / math.sqrt(float(np.sum(sk * sk)))
    Vk = V[:, :k]
    mps.B[n0] = (C.reshape(2 * Dl, 2 * Dr) @ Vk).reshape(Dl, 2, k)
    mps.B[n0 + 1] = Vk.conj().T.reshape(k, 2, Dr)
    mps.lam[n0] = lam_new
    if keep_tape:
        return dict(bond=n0, Bl=Bl, Br=Br, lam_left=lam_left, G=G, C=C, Cm=Cm, s=s, V=V, k=k,
                    lam_new=lam_new)
    return None


def apply_circuit(mps: MPS, gates, theta, D: int, eps: float, phi_override=None):
    """U(theta)|mps>, gates in time order (Sec. 4, Eq. pqc)."""
    for t, g in enumerate(gates):
        phi = None if phi_override is None else phi_override.get(t)
        apply_gate(mps, g.bond, g.matrix(theta, phi=phi), D, eps)
    return mps


# ---- contractions ----------------------------------------------------------------

# The sums over bond indices below are written as matrix products of reshaped tensors (the
# same contractions; a library matmul is one step), the 2x2 operator on the physical index as
# an einsum.

def two_site(Bl, Br):
    """Theta[a, i, j, c] = sum_m Bl[a, i, m] Br[m, j, c]."""
    Dl, _, Dm = Bl.shape
    Dr = Br.shape[2]
    return (Bl.reshape(2 * Dl, Dm) @ Br.reshape(Dm, 2 * Dr)).reshape(Dl, 2, 2, Dr)


def transfer_left(L, B, O):
    """L'[b', b] = sum conj(B[a', i', b']) O[i', i] L[a', a] B[a, i, b]."""
    Dl, _, Dr = B.shape
    T = (L @ B.reshape(Dl, 2 * Dr)).reshape(L.shape[0], 2, Dr)      # sum_a L[a', a] B[a, i, b]
    T = np.einsum("ji,xib->xjb", O, T)                               # O on the physical index
    return B.reshape(2 * Dl, Dr).conj().T @ T.reshape(2 * Dl, Dr)    # sum_{a', i'} conj(B[a', i', b'])


def transfer_right(R, B, O):
    """R'[a', a] = sum conj(B[a', i', b']) O[i', i] B[a, i, b] R[b', b]."""
    Dl, _, Dr = B.shape
    T = (B.reshape(2 * Dl, Dr) @ R.T).reshape(Dl, 2, R.shape[0])     # sum_b B[a, i, b] R[b', b]
    T = np.einsum("ji,aiy->ajy", O, T)
    return B.reshape(Dl, 2 * Dr).conj() @ T.reshape(Dl, 2 * Dr).T   # sum_{i', b'} conj(B[a', i', b'])


def site_env(L, O, B, R):
    """d<psi|O|psi>/d conj(B[a', i', b']) = sum L[a', a] O[i', i] B[a, i, b] R[b', b]."""
    Dl, _, Dr = B.shape
    T = (L @ B.reshape(Dl, 2 * Dr)).reshape(L.shape[0], 2, Dr)
    T = np.einsum("ji,xib->xjb", O, T)
    return (T.reshape(-1, Dr) @ R.T).reshape(L.shape[0], 2, R.shape[0])


def identity_envs(mps: MPS):
    """L^I_s (sites 0..s contracted) and R^I_s (sites s..n-1); L[-1] = R[n] = [[1]]."""
    n = mps.n
    I = np.eye(2, dtype=complex)
    L = [None] * n
    R = [None] * (n + 1)
    cur = np.ones((1, 1), dtype=complex)
    for s in range(n):
        cur = transfer_left(cur, mps.B[s], I)
        L[s] = cur
    R[n] = np.ones((1, 1), dtype=complex)
    for s in range(n - 1, -1, -1):
        R[s] = transfer_right(R[s + 1], mps.B[s], I)
    return L, R


def left_of(Lid, s):
    return np.ones((1, 1), dtype=complex) if s < 0 else Lid[s]


def string_expectations(mps: MPS, ham: pauli.PauliHamiltonian):
    """e_k = <psi|P_k|psi> (Eq. paulistringexp) and Z = <psi|psi>.

    Each string is contracted over its support [a, b] between the identity
    environments L^I_{a-1} and R^I_{b+1}; outside the support the network is the
    identity network, so this is the full contraction.
    """
    Lid, Rid = identity_envs(mps)
    Z = Lid[mps.n - 1][0, 0]
    e = np.zeros(len(ham), dtype=complex)
    for k, (x, z) in enumerate(zip(ham.x, ham.z)):
        a, b = pauli.support_range(x, z)
        if a < 0:
            e[k] = Z
            continue
        L = left_of(Lid, a - 1)
        for s in range(a, b + 1):
            L = transfer_left(L, mps.B[s], pauli.site_matrix(x, z, s))
        e[k] = np.sum(L * Rid[b + 1])
    return e, Z


def energy(mps: MPS, ham: pauli.PauliHamiltonian) -> float:
    """E = sum_k c_k Re e_k / Z (Eq. expect-val, normalised)."""
    e, Z = string_expectations(mps, ham)
    return math.fsum(ham.coeff * e.real) / Z.real


def energy_seed(mps: MPS, ham: pauli.PauliHamiltonian):
    """E and Bbar_s = dE/d conj(B_s) = [sum_k c_k env_k(s) - E env_I(s)] / Z.

    env_k(s) is the network of <psi|P_k|psi> with conj(B_s) removed (Eq. expecgrad:
    the derivative of <psi|H|psi> with respect to <psi| is H|psi>); every string's
    left and right environments are contracted in full, site by site.
    """
    n = mps.n
    e, Z = string_expectations(mps, ham)
    Zr = Z.real
    E = math.fsum(ham.coeff * e.real) / Zr
    Lid, Rid = identity_envs(mps)
    I = np.eye(2, dtype=complex)
    Bbar = [np.zeros_like(b) for b in mps.B]
    for s in range(n):
        env_I = site_env(left_of(Lid, s - 1), I, mps.B[s], Rid[s + 1])
        Bbar[s] -= E * env_I
    for k, (x, z, c) in enumerate(zip(ham.x, ham.z, ham.coeff)):
        ops = [pauli.site_matrix(x, z, s) for s in range(n)]
        Ls = [None] * n                    # Ls[s] = left env after site s
        cur = np.ones((1, 1), dtype=complex)
        for s in range(n):
            cur = transfer_left(cur, mps.B[s], ops[s])
            Ls[s] = cur
        Rs = [None] * (n + 1)
        Rs[n] = np.ones((1, 1), dtype=complex)
        for s in range(n - 1, -1, -1):
            Rs[s] = transfer_right(Rs[s + 1], mps.B[s], ops[s])
        for s in range(n):
            Lm = np.ones((1, 1), dtype=complex) if s == 0 else Ls[s - 1]
            Bbar[s] += c * site_env(Lm, ops[s], mps.B[s], Rs[s + 1])
    Bbar = [b / Zr for b in Bbar]
    return E, Bbar


# ---- reverse pass ------------------------------------------------------------------

def svd_adjoint(Cm, s, V, k, sbar_k, Vbar_k):
    """Cotangent of C~ given sbar (kept) and Vbar (kept columns); U is not used.

    M = C~^+ C~ = V diag(w) V^+, w = s^2 padded with zeros to the column count.
    dE = sum wbar dw + 2 Re <Vbar, dV> gives, with J = F o (V^+ Vbar),
    Mbar = V (diag(wbar) + J + J^+) V^+ (Hermitian, dE = tr(Mbar dM)) and
    C~bar = C~ Mbar = (C~ V)(diag(wbar) + J + J^+) V^+, where the columns of C~ V that
    belong to numerical zeros (s_i <= NULL_REL s_1) are set to zero.
    """
    ncol = V.shape[0]
    w = np.zeros(ncol)
    w[: len(s)] = s * s
    sv = np.zeros(ncol)
    sv[: len(s)] = s
    null = np.ones(ncol, dtype=bool)
    null[: len(s)] = s <= NULL_REL * s[0]
    w[null] = 0.0
    sv[null] = 0.0
    wbar = np.zeros(ncol)
    wbar[:k] = sbar_k / (2.0 * s[:k])
    Vbar = np.zeros((ncol, ncol), dtype=complex)
    Vbar[:, :k] = Vbar_k
    dw = w[None, :] - w[:, None]                  # dw[i, j] = w_j - w_i
    big = (np.abs(dw) > DEGEN_REL * np.maximum(w[None, :], w[:, None])) & \
          (np.abs(sv[None, :] - sv[:, None]) > DEGEN_ABS * s[0])
    F = np.where(big, 1.0 / np.where(big, dw, 1.0), 0.0)   # diagonal: dw = 0 -> 0
    J = F * (V.conj().T @ Vbar)
    W = Cm @ V
    W[:, null] = 0.0
    return W @ (np.diag(wbar) + J + J.conj().T) @ V.conj().T


def gate_adjoint(tape, Bbar_l_new, Bbar_r_new, lambar_new, dG):
    """Reverse of one gate.  Returns (Bbar_l, Bbar_r, lambar_left contribution, dE/dphi)."""
    Bl, Br, C, Cm, s, V, k = (tape[q] for q in ("Bl", "Br", "C", "Cm", "s", "V", "k"))
    lam_left, G, lam_new = tape["lam_left"], tape["G"], tape["lam_new"]
    Dl, Dr = Bl.shape[0], Br.shape[2]
    Vk = V[:, :k]
    Cu = C.reshape(2 * Dl, 2 * Dr)
    bl = Bbar_l_new.reshape(2 * Dl, k)
    br = Bbar_r_new.reshape(k, 2 * Dr)
    # B~_{n+1} = Vk^+ ; B~_n = C Vk
    Vbar_k = br.conj().T + Cu.conj().T @ bl
    Cbar = bl @ Vk.conj().T
    # lambda~ = s_k / ||s_k||
    nrm = math.sqrt(float(np.sum(s[:k] ** 2)))
    sbar_k = (lambar_new - lam_new * float(np.dot(lam_new, lambar_new))) / nrm
    Ctbar = svd_adjoint(Cm, s, V, k, sbar_k, Vbar_k).reshape(Dl, 2, 2, Dr)
    Cbar = Cbar.reshape(Dl, 2, 2, Dr) + lam_left[:, None, None, None] * Ctbar
    lambar_left = 2.0 * np.real(np.einsum("aijc,aijc->a", Ctbar.conj(), C))
    theta4 = two_site(Bl, Br).reshape(Dl, 4, Dr)
    Cb4 = Cbar.reshape(Dl, 4, Dr)
    Gbar = np.einsum("axc,ayc->xy", Cb4, theta4.conj())
    dphi = 2.0 * float(np.real(np.sum(Gbar.conj() * dG)))
    Thbar = np.einsum("xy,axc->ayc", G.conj(), Cb4).reshape(Dl, 2, 2, Dr)
    Dm = Bl.shape[2]
    Th2 = Thbar.reshape(2 * Dl, 2 * Dr)
    Bbar_l = (Th2 @ Br.reshape(Dm, 2 * Dr).conj().T).reshape(Dl, 2, Dm)   # sum_{j,c} Thbar conj(Br)
    Bbar_r = (Bl.reshape(2 * Dl, Dm).conj().T @ Th2).reshape(Dm, 2, Dr)   # sum_{a,i} conj(Bl) Thbar
    return Bbar_l, Bbar_r, lambar_left, dphi


@dataclass
class GradResult:
    E: float
    grad: np.ndarray
    gate_grad: np.ndarray
    final: MPS = None
    kept: list = field(default_factory=list)


def energy_grad(mps0: MPS, gates, theta, ham, D: int, eps: float, checkpoint_every: int = 512,
                phi_override=None) -> GradResult:
    """E(theta) of U(theta)|mps0> and dE/dtheta by reverse mode through the truncated forward.

    The forward keeps an MPS snapshot every `checkpoint_every` gates; the reverse pass
    walks the segments backwards, re-running each segment's forward with a tape
    (memory: snapshots + one segment of tapes, Sec. 4's point about not storing every
    intermediate state).
    """
    theta = np.asarray(theta, dtype=float)
    ng = len(gates)
    K = max(1, checkpoint_every)
    mats = []
    dmats = []
    for t, g in enumerate(gates):
        phi = None if phi_override is None else phi_override.get(t)
        mats.append(g.matrix(theta, phi=phi))
        dmats.append(g.dmatrix(theta, phi=phi))
    mps = mps0.copy()
    snaps = []
    for t, g in enumerate(gates):
        if t % K == 0:
            snaps.append(mps.copy())
        apply_gate(mps, g.bond, mats[t], D, eps)
    E, Bbar = energy_seed(mps, ham)
    lambar = [np.zeros_like(l) for l in mps.lam]
    gate_grad = np.zeros(ng)
    for seg in range((ng + K - 1) // K - 1, -1, -1):
        lo, hi = seg * K, min(ng, (seg + 1) * K)
        cur = snaps[seg].copy()
        tapes = [apply_gate(cur, gates[t].bond, mats[t], D, eps, keep_tape=True) for t in range(lo, hi)]
        for t in range(hi - 1, lo - 1, -1):
            b = gates[t].bond
            bl, br, lbl, dphi = gate_adjoint(tapes[t - lo], Bbar[b], Bbar[b + 1], lambar[b], dmats[t])
            Bbar[b], Bbar[b + 1] = bl, br
            lambar[b] = np.zeros(bl.shape[2])
            if b > 0:
                lambar[b - 1] = lambar[b - 1] + lbl
            gate_grad[t] = dphi
    grad = np.zeros(len(theta))
    for t, g in enumerate(gates):
        if g.parametric:
            grad[g.theta_idx] += g.scale * gate_grad[t]
    return GradResult(E=E, grad=grad, gate_grad=gate_grad, final=mps)


def regauge(mps: MPS, bond: int, X: np.ndarray) -> MPS:
    """B_bond -> B_bond X, B_{bond+1} -> X^-1 B_{bond+1} (leaves the state unchanged)."""
    out = mps.copy()
    out.B[bond] = np.einsum("aim,mk->aik", out.B[bond], X)
    out.B[bond + 1] = np.einsum("km,mjc->kjc", np.linalg.inv(X), out.B[bond + 1])
    return out


def to_dense(mps: MPS) -> np.ndarray:
    """Contract the MPS into the 2^n coefficient vector (site 0 most significant)."""
    v = mps.B[0].reshape(2, -1)
    for b in mps.B[1:]:
        v = np.einsum("pm,mjc->pjc", v, b).reshape(-1, b.shape[2])
    return v.reshape(-1)


def right_canonical_residual(mps: MPS) -> float:
    """max_s || sum_i B^i B^i+ - I || (Eq. rightcanonicalcondition)."""
    worst = 0.0
    for b in mps.B:
        Dl = b.shape[0]
        m = b.reshape(Dl, -1)
        worst = max(worst, float(np.abs(m @ m.conj().T - np.eye(Dl)).max()))
    return worst

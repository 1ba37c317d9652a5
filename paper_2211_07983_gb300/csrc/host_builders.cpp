// Host-side problem builders (step S0): Jordan-Wigner qubit Hamiltonian and the UCC
// circuit compiler.  Plain C++17, no CUDA; built into libmps.
//
// Hamiltonian: Sec. 2, Eq. (ham-pbc) read in chemist notation,
//   H = sum_pq h_pq a+_p a_q + 1/2 sum_pqrs (pq|rs) a+_p a+_r a_s a_q,
// Jordan-Wigner a_p = Z_0..Z_{p-1} (X_p + i Y_p)/2 with |1> = occupied (Eq. expect-val).
// Circuit: Sec. 2 (UCC ansatz, first-order Trotter, "V-shaped" blocks) and Sec. 3
// (gate fusion); the rules are spelled out in mps_compile_excitations below.
#include <algorithm>
#include <array>
#include <cmath>
#include <complex>
#include <cstring>
#include <map>
#include <unordered_map>
#include <utility>
#include <vector>

#include "mps_internal.h"

namespace {

using cd = std::complex<double>;

// ---- single-qubit Pauli algebra -------------------------------------------------------
// Symbols: 0 = I, 1 = X, 2 = Y, 3 = Z.  (x, z) bits: X (1,0), Y (1,1), Z (0,1).
inline int sym_of(uint64_t x, uint64_t z, int s) {
  int xb = (x >> s) & 1, zb = (z >> s) & 1;
  return xb ? (zb ? 2 : 1) : (zb ? 3 : 0);
}

// Product table A*B = i^p C for non-identity A, B: returns p (C follows from xor).
//            X  Y  Z   (column = right factor)
// X:         0  1  3   (XX = I, XY = iZ, XZ = -iY)
// Y:         3  0  1   (YX = -iZ, YY = I, YZ = iX)
// Z:         1  3  0   (ZX = iY, ZY = -iX, ZZ = I)
constexpr int kPhase[3][3] = {{0, 1, 3}, {3, 0, 1}, {1, 3, 0}};

struct PTerm {   // i^k * P(x, z)
  int k;
  uint64_t x, z;
};

inline PTerm pmul(const PTerm& a, const PTerm& b) {
  uint64_t both = (a.x | a.z) & (b.x | b.z);
  int k = a.k + b.k;
  while (both) {
    int s = __builtin_ctzll(both);
    both &= both - 1;
    k += kPhase[sym_of(a.x, a.z, s) - 1][sym_of(b.x, b.z, s) - 1];
  }
  return PTerm{k & 3, a.x ^ b.x, a.z ^ b.z};
}

// a_p = 1/2 Z_<p X_p + i/2 Z_<p Y_p ; a+_p = 1/2 Z_<p X_p - i/2 Z_<p Y_p (weights 1/2 implied)
inline std::array<PTerm, 2> annihilate(int p) {
  uint64_t below = (p == 0) ? 0ull : ((1ull << p) - 1ull);
  uint64_t e = 1ull << p;
  return {PTerm{0, e, below}, PTerm{1, e, below | e}};
}
inline std::array<PTerm, 2> create(int p) {
  uint64_t below = (p == 0) ? 0ull : ((1ull << p) - 1ull);
  uint64_t e = 1ull << p;
  return {PTerm{0, e, below}, PTerm{3, e, below | e}};
}

// ---- exact summation ------------------------------------------------------------------
// Shewchuk's non-overlapping expansion (grow-expansion with Knuth's TwoSum) plus a final
// correctly rounded (round-half-even) collapse.  The merged coefficient is therefore the
// correctly rounded value of the exact sum, independent of the order of contributions.
struct Expansion {
  std::vector<double> p;  // increasing magnitude, non-overlapping
  void add(double x) {
    size_t i = 0;
    for (size_t j = 0; j < p.size(); ++j) {
      double y = p[j];
      if (std::fabs(x) < std::fabs(y)) std::swap(x, y);
      double hi = x + y;
      double lo = y - (hi - x);
      if (lo != 0.0) p[i++] = lo;
      x = hi;
    }
    p.resize(i);
    p.push_back(x);
  }
  double value() const {
    if (p.empty()) return 0.0;
    size_t n = p.size();
    double hi = p[--n];
    double lo = 0.0;
    while (n > 0) {
      double x = hi;
      double y = p[--n];
      hi = x + y;
      double yr = hi - x;
      lo = y - yr;
      if (lo != 0.0) break;
    }
    // round-half-even across the remaining (smaller) components
    if (n > 0 && ((lo < 0.0 && p[n - 1] < 0.0) || (lo > 0.0 && p[n - 1] > 0.0))) {
      double y = lo * 2.0;
      double x = hi + y;
      double yr = x - hi;
      if (y == yr) hi = x;
    }
    return hi;
  }
};

struct KeyHash {
  size_t operator()(const std::pair<uint64_t, uint64_t>& k) const {
    return std::hash<uint64_t>()(k.first * 0x9E3779B97F4A7C15ull ^ (k.second + 0x632BE59BD9B4E019ull));
  }
};

struct Accumulator {
  std::unordered_map<std::pair<uint64_t, uint64_t>, std::pair<Expansion, Expansion>, KeyHash> m;
  // contribution value * i^k
  void add(const PTerm& t, double value) {
    if (value == 0.0) return;
    auto& e = m[{t.x, t.z}];
    switch (t.k) {
      case 0: e.first.add(value); break;
      case 1: e.second.add(value); break;
      case 2: e.first.add(-value); break;
      default: e.second.add(-value); break;
    }
  }
};

// Expand a product of single-mode operators (each a 2-term sum) into Pauli terms.
template <size_t N>
void expand(const std::array<std::array<PTerm, 2>, N>& f, std::vector<PTerm>& out) {
  out.clear();
  out.push_back(PTerm{0, 0, 0});
  for (size_t q = 0; q < N; ++q) {
    std::vector<PTerm> nxt;
    nxt.reserve(out.size() * 2);
    for (const auto& t : out)
      for (const auto& u : f[q]) nxt.push_back(pmul(t, u));
    out.swap(nxt);
  }
}

// Canonical order: identity first; then first non-identity site a; then symbols from a up
// (I < X < Y < Z).
struct Canon {
  int n;
  static int first_site(uint64_t x, uint64_t z) {
    uint64_t s = x | z;
    return s ? __builtin_ctzll(s) : -1;
  }
  bool operator()(const std::pair<uint64_t, uint64_t>& A, const std::pair<uint64_t, uint64_t>& B) const {
    int a1 = first_site(A.first, A.second), a2 = first_site(B.first, B.second);
    if (a1 != a2) return a1 < a2;
    if (a1 < 0) return false;
    for (int s = a1; s < n; ++s) {
      int u = sym_of(A.first, A.second, s), v = sym_of(B.first, B.second, s);
      if (u != v) return u < v;
    }
    return false;
  }
};

struct Merged {
  uint64_t x, z;
  double re, im;
};

std::vector<Merged> merge(const Accumulator& acc, int n, double drop_rel, bool* nonhermitian) {
  std::vector<Merged> all;
  all.reserve(acc.m.size());
  double cmax = 0.0;
  for (const auto& kv : acc.m) {
    Merged g{kv.first.first, kv.first.second, kv.second.first.value(), kv.second.second.value()};
    cmax = std::max(cmax, std::hypot(g.re, g.im));
    all.push_back(g);
  }
  std::vector<Merged> keep;
  *nonhermitian = false;
  for (const auto& g : all) {
    if (std::hypot(g.re, g.im) <= drop_rel * cmax) continue;
    if (std::fabs(g.im) > drop_rel * cmax) *nonhermitian = true;
    keep.push_back(g);
  }
  Canon cmp{n};
  std::sort(keep.begin(), keep.end(), [&](const Merged& a, const Merged& b) {
    return cmp({a.x, a.z}, {b.x, b.z});
  });
  return keep;
}

// ---- circuit compiler -----------------------------------------------------------------
enum Kind : int { K_H = 0, K_RXP, K_RXM, K_RZ, K_CNOT, K_SWAP, K_ID };

struct Prim {
  int kind;
  int q;          // 1q: qubit; 2q: bond (lower site)
  int theta_idx;  // RZ only
  double scale;   // RZ only
  bool two() const { return kind >= K_CNOT; }
};

using M4 = std::array<cd, 16>;
using M2 = std::array<cd, 4>;

M4 eye4() {
  M4 m{};
  for (int i = 0; i < 4; ++i) m[i * 4 + i] = 1.0;
  return m;
}
M4 mul4(const M4& a, const M4& b) {  // a @ b
  M4 c{};
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      cd acc = 0.0;
      for (int k = 0; k < 4; ++k) acc += a[i * 4 + k] * b[k * 4 + j];
      c[i * 4 + j] = acc;
    }
  return c;
}
M4 kron_low(const M2& w) {  // w (x) I : acts on the lower site (major index)
  M4 m{};
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b)
      for (int t = 0; t < 2; ++t) m[(2 * a + t) * 4 + (2 * b + t)] = w[a * 2 + b];
  return m;
}
M4 kron_high(const M2& w) {  // I (x) w
  M4 m{};
  for (int t = 0; t < 2; ++t)
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) m[(2 * t + a) * 4 + (2 * t + b)] = w[a * 2 + b];
  return m;
}
M2 one_q(int kind) {
  const double r = 1.0 / std::sqrt(2.0);
  switch (kind) {
    case K_H: return {cd(r), cd(r), cd(r), cd(-r)};
    case K_RXP: return {cd(r), cd(0, -r), cd(0, -r), cd(r)};   // Rx(+pi/2) = (I - iX)/sqrt2
    default: return {cd(r), cd(0, r), cd(0, r), cd(r)};        // Rx(-pi/2)
  }
}
M4 two_q(int kind) {
  M4 m{};
  if (kind == K_CNOT) {  // control = lower site
    m[0] = m[5] = 1.0;
    m[2 * 4 + 3] = m[3 * 4 + 2] = 1.0;
  } else if (kind == K_SWAP) {
    m[0] = m[15] = 1.0;
    m[1 * 4 + 2] = m[2 * 4 + 1] = 1.0;
  } else {
    m = eye4();
  }
  return m;
}

struct Fused {
  int bond;
  int theta_idx = -1;
  double scale = 0.0;
  int rz_site = 0;
  M4 mat, pre, post;
};

bool inverse_pair(const Prim& h, const Prim& g) {
  if (h.two() != g.two() || h.q != g.q) return false;
  if (!g.two()) {
    if (g.kind == K_RZ || h.kind == K_RZ) return false;
    return (h.kind == K_H && g.kind == K_H) || (h.kind == K_RXP && g.kind == K_RXM) ||
           (h.kind == K_RXM && g.kind == K_RXP);
  }
  return h.kind == g.kind && (g.kind == K_CNOT || g.kind == K_SWAP);
}

}  // namespace

extern "C" mps_status mps_build_hamiltonian(int32_t n, const double* h, const double* eri,
                                            int64_t capacity, uint64_t* x_mask, uint64_t* z_mask,
                                            double* coeff, int64_t* n_terms_out) {
  mpsi::clear_error();
  if (n < 1 || n > 64) return mpsi::fail(MPS_EINVAL, "mps_build_hamiltonian: n must be in 1..64");
  if (!h || !eri || !n_terms_out) return mpsi::fail(MPS_EINVAL, "mps_build_hamiltonian: null pointer");
  Accumulator acc;
  std::vector<PTerm> terms;
  for (int p = 0; p < n; ++p)
    for (int q = 0; q < n; ++q) {
      double v = h[(size_t)p * n + q];
      if (v == 0.0) continue;
      if (!std::isfinite(v)) return mpsi::fail(MPS_EINVAL, "mps_build_hamiltonian: non-finite h");
      expand<2>({create(p), annihilate(q)}, terms);
      for (const auto& t : terms) acc.add(t, v * 0.25);
    }
  const size_t nn = (size_t)n;
  for (size_t p = 0; p < nn; ++p)
    for (size_t q = 0; q < nn; ++q)
      for (size_t r = 0; r < nn; ++r)
        for (size_t s = 0; s < nn; ++s) {
          double v = eri[((p * nn + q) * nn + r) * nn + s];
          if (v == 0.0 || p == r || q == s) continue;  // a+_p a+_p = a_s a_s = 0
          if (!std::isfinite(v)) return mpsi::fail(MPS_EINVAL, "mps_build_hamiltonian: non-finite eri");
          expand<4>({create((int)p), create((int)r), annihilate((int)s), annihilate((int)q)}, terms);
          for (const auto& t : terms) acc.add(t, v * 0.03125);  // 1/2 * 2^-4
        }
  bool nonherm = false;
  auto keep = merge(acc, n, 1e-14, &nonherm);
  if (nonherm) return mpsi::fail(MPS_EINVAL, "mps_build_hamiltonian: integrals give a non-Hermitian H");
  *n_terms_out = (int64_t)keep.size();
  if ((int64_t)keep.size() > capacity || !x_mask || !z_mask || !coeff)
    return mpsi::fail(MPS_EINVAL, "mps_build_hamiltonian: output capacity too small");
  for (size_t t = 0; t < keep.size(); ++t) {
    x_mask[t] = keep[t].x;
    z_mask[t] = keep[t].z;
    coeff[t] = keep[t].re;
  }
  return MPS_OK;
}

// Compilation rules (Sec. 2 V-shaped blocks, Sec. 3 fusion):
//  * generator T - T+ (T = a+_a a_i, or a+_a a+_b a_j a_i) -> sum_P (i c_P) P, strings in
//    canonical order; exp(i theta c P) = exp(-i phi/2 P) with phi = -2 c theta.
//  * block: basis change on X (H) / Y (Rx(+pi/2)) sites, ladder over [a, b) with
//    CNOT(s -> s+1) if site s+1 is non-identity else SWAP(s, s+1), Rz(phi) on b, ladder
//    reversed, basis change back (H / Rx(-pi/2)).
//  * (1) cancel adjacent inverse pairs with per-qubit stacks; (2) absorb 1q gates into the
//    next 2q gate touching their qubit, else the previous one; (3) merge same-bond runs
//    (at most one Rz angle per fused gate).
extern "C" mps_status mps_compile_excitations(int32_t n, const int32_t* exc, int32_t n_exc,
                                              int64_t capacity, mps_gate* gates_out,
                                              int64_t* n_gates_out) {
  mpsi::clear_error();
  if (n < 2 || n > 64) return mpsi::fail(MPS_EINVAL, "mps_compile_excitations: n must be in 2..64");
  if (n_exc < 0 || (n_exc > 0 && !exc) || !n_gates_out)
    return mpsi::fail(MPS_EINVAL, "mps_compile_excitations: bad arguments");
  std::vector<Prim> prims;
  std::vector<PTerm> terms;
  for (int t = 0; t < n_exc; ++t) {
    int i = exc[4 * t], j = exc[4 * t + 1], a = exc[4 * t + 2], b = exc[4 * t + 3];
    bool single = (j < 0);
    auto in_range = [&](int v) { return v >= 0 && v < n; };
    if (!in_range(i) || !in_range(a) || (!single && (!in_range(j) || !in_range(b))) || (single && b >= 0))
      return mpsi::fail(MPS_EINVAL, "mps_compile_excitations: orbital index out of range");
    Accumulator acc;
    if (single) {
      expand<2>({create(a), annihilate(i)}, terms);
      for (const auto& u : terms) acc.add(u, 0.25);
      expand<2>({create(i), annihilate(a)}, terms);
      for (const auto& u : terms) acc.add(u, -0.25);
    } else {
      expand<4>({create(a), create(b), annihilate(j), annihilate(i)}, terms);
      for (const auto& u : terms) acc.add(u, 0.0625);
      expand<4>({create(i), create(j), annihilate(b), annihilate(a)}, terms);
      for (const auto& u : terms) acc.add(u, -0.0625);
    }
    bool nonherm = false;
    auto strings = merge(acc, n, 0.0, &nonherm);  // all nonzero strings; coefficients i*c
    for (const auto& st : strings) {
      if (st.re != 0.0 || st.im == 0.0)
        return mpsi::fail(MPS_EINVAL, "mps_compile_excitations: generator is not anti-Hermitian");
      double scale = -2.0 * st.im;
      int lo = __builtin_ctzll(st.x | st.z), hi = 63 - __builtin_clzll(st.x | st.z);
      for (int s = lo; s <= hi; ++s) {
        int y = sym_of(st.x, st.z, s);
        if (y == 1) prims.push_back({K_H, s, -1, 0.0});
        if (y == 2) prims.push_back({K_RXP, s, -1, 0.0});
      }
      std::vector<Prim> ladder;
      for (int s = lo; s < hi; ++s)
        ladder.push_back({sym_of(st.x, st.z, s + 1) != 0 ? K_CNOT : K_SWAP, s, -1, 0.0});
      prims.insert(prims.end(), ladder.begin(), ladder.end());
      prims.push_back({K_RZ, hi, t, scale});
      prims.insert(prims.end(), ladder.rbegin(), ladder.rend());
      for (int s = lo; s <= hi; ++s) {
        int y = sym_of(st.x, st.z, s);
        if (y == 1) prims.push_back({K_H, s, -1, 0.0});
        if (y == 2) prims.push_back({K_RXM, s, -1, 0.0});
      }
    }
  }
  // (1) cancellation
  std::vector<Prim> kept;
  std::vector<char> alive;
  std::vector<std::vector<int>> stk(n);
  for (const auto& g : prims) {
    int q0 = g.q, q1 = g.two() ? g.q + 1 : -1;
    int top = stk[q0].empty() ? -1 : stk[q0].back();
    bool ok = top >= 0 && (q1 < 0 || (!stk[q1].empty() && stk[q1].back() == top)) &&
              kept[top].two() == g.two() && kept[top].q == g.q && inverse_pair(kept[top], g);
    if (ok) {
      stk[q0].pop_back();
      if (q1 >= 0) stk[q1].pop_back();
      alive[top] = 0;
      continue;
    }
    kept.push_back(g);
    alive.push_back(1);
    stk[q0].push_back((int)kept.size() - 1);
    if (q1 >= 0) stk[q1].push_back((int)kept.size() - 1);
  }
  std::vector<Prim> p1;
  for (size_t u = 0; u < kept.size(); ++u)
    if (alive[u]) p1.push_back(kept[u]);
  // a qubit never touched by a two-qubit gate gets an identity two-qubit gate at its first use
  {
    std::vector<char> touched(n, 0);
    for (const auto& g : p1)
      if (g.two()) touched[g.q] = touched[g.q + 1] = 1;
    std::vector<Prim> p2;
    for (const auto& g : p1) {
      if (!g.two() && !touched[g.q]) {
        int bnd = g.q < n - 1 ? g.q : g.q - 1;
        p2.push_back({K_ID, bnd, -1, 0.0});
        touched[bnd] = touched[bnd + 1] = 1;
      }
      p2.push_back(g);
    }
    p1.swap(p2);
  }
  // (2) absorption: for each 1q gate find the next 2q gate on its qubit, else the previous
  const int np = (int)p1.size();
  std::vector<int> next2(np, -1), prev2(np, -1);
  {
    std::vector<int> last(n, -1);
    for (int u = 0; u < np; ++u) {
      if (p1[u].two()) {
        last[p1[u].q] = last[p1[u].q + 1] = u;
      } else {
        prev2[u] = last[p1[u].q];
      }
    }
    std::fill(last.begin(), last.end(), -1);
    for (int u = np - 1; u >= 0; --u) {
      if (p1[u].two()) {
        last[p1[u].q] = last[p1[u].q + 1] = u;
      } else {
        next2[u] = last[p1[u].q];
      }
    }
  }
  std::vector<std::vector<int>> before(np), after(np);
  for (int u = 0; u < np; ++u) {
    if (p1[u].two()) continue;
    if (next2[u] >= 0)
      before[next2[u]].push_back(u);
    else
      after[prev2[u]].push_back(u);
  }
  std::vector<Fused> fused;
  for (int u = 0; u < np; ++u) {
    if (!p1[u].two()) continue;
    const int bond = p1[u].q;
    std::vector<int> seq(before[u]);
    seq.push_back(-1 - u);  // marker for the 2q core
    seq.insert(seq.end(), after[u].begin(), after[u].end());
    int rz_pos = -1;
    for (size_t v = 0; v < seq.size(); ++v)
      if (seq[v] >= 0 && p1[seq[v]].kind == K_RZ) {
        if (rz_pos >= 0) return mpsi::fail(MPS_EINVAL, "mps_compile_excitations: two Rz angles in one gate");
        rz_pos = (int)v;
      }
    auto mat_of = [&](int e) -> M4 {
      if (e < 0) return two_q(p1[-1 - e].kind);
      const Prim& g = p1[e];
      return g.q == bond ? kron_low(one_q(g.kind)) : kron_high(one_q(g.kind));
    };
    auto prod = [&](size_t from, size_t to) {  // time order [from, to)
      M4 m = eye4();
      for (size_t v = from; v < to; ++v) m = mul4(mat_of(seq[v]), m);
      return m;
    };
    Fused f;
    f.bond = bond;
    if (rz_pos < 0) {
      f.mat = prod(0, seq.size());
    } else {
      const Prim& r = p1[seq[rz_pos]];
      f.theta_idx = r.theta_idx;
      f.scale = r.scale;
      f.rz_site = (r.q == bond) ? 0 : 1;
      f.pre = prod(0, rz_pos);
      f.post = prod(rz_pos + 1, seq.size());
    }
    fused.push_back(f);
  }
  // (3) merge same-bond runs
  std::vector<Fused> out;
  std::vector<int> last(n, -1);
  for (auto& g : fused) {
    int lo = g.bond, hi = g.bond + 1;
    int t = last[lo];
    if (t >= 0 && last[hi] == t && out[t].bond == g.bond &&
        !(out[t].theta_idx >= 0 && g.theta_idx >= 0)) {
      Fused& h = out[t];
      if (h.theta_idx < 0 && g.theta_idx < 0) {
        h.mat = mul4(g.mat, h.mat);
      } else if (h.theta_idx >= 0) {
        h.post = mul4(g.mat, h.post);
      } else {
        Fused nf = g;
        nf.pre = mul4(g.pre, h.mat);
        h = nf;
      }
      continue;
    }
    out.push_back(g);
    last[lo] = last[hi] = (int)out.size() - 1;
  }
  *n_gates_out = (int64_t)out.size();
  if ((int64_t)out.size() > capacity || !gates_out)
    return mpsi::fail(MPS_EINVAL, "mps_compile_excitations: output capacity too small");
  for (size_t u = 0; u < out.size(); ++u) {
    mps_gate& g = gates_out[u];
    std::memset(&g, 0, sizeof(g));
    g.bond = out[u].bond;
    g.theta_idx = out[u].theta_idx;
    g.rz_site = out[u].rz_site;
    g.theta_scale = out[u].scale;
    auto put = [](double* dst, const M4& m) {
      for (int e = 0; e < 16; ++e) {
        dst[2 * e] = m[e].real();
        dst[2 * e + 1] = m[e].imag();
      }
    };
    if (g.theta_idx < 0) {
      put(g.mat, out[u].mat);
    } else {
      put(g.pre, out[u].pre);
      put(g.post, out[u].post);
    }
  }
  return MPS_OK;
}

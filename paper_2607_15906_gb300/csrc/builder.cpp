// Host build of the method's tables (runs once per Hamiltonian, not timed):
//   integrals -> Eq. (2) fermionic H -> Eq. (3) Pauli sum under JW or BK
//   (Sec. II.A), the spin-conserving singles+doubles pool (Table II), and
//   Greedy Operator Commutativity Partitioning of the pool (Sec. III.A,
//   Algorithm 1).
#include <algorithm>
#include <cmath>
#include <numeric>

#include "internal.h"

namespace gocp {

namespace {

inline int parity32(uint32_t v) { return __builtin_popcount(v) & 1; }

// GF(2) inverse of a lower-triangular-or-not matrix given as row masks.
std::vector<uint32_t> gf2_inverse_rows(const std::vector<uint32_t>& rows, int n) {
  std::vector<uint32_t> a(rows), inv(n);
  for (int i = 0; i < n; ++i) inv[i] = 1u << i;
  for (int c = 0; c < n; ++c) {
    int piv = -1;
    for (int r = c; r < n; ++r)
      if ((a[r] >> c) & 1u) { piv = r; break; }
    if (piv < 0) return {};
    std::swap(a[c], a[piv]);
    std::swap(inv[c], inv[piv]);
    for (int r = 0; r < n; ++r)
      if (r != c && ((a[r] >> c) & 1u)) { a[r] ^= a[c]; inv[r] ^= inv[c]; }
  }
  return inv;
}

// y = M v over GF(2) with M given by rows.
uint32_t apply_rows(const std::vector<uint32_t>& rows, uint32_t v) {
  uint32_t out = 0;
  for (size_t i = 0; i < rows.size(); ++i) out |= (uint32_t)parity32(rows[i] & v) << i;
  return out;
}

// Rows of M^T from rows of M.
std::vector<uint32_t> transpose_rows(const std::vector<uint32_t>& rows, int n) {
  std::vector<uint32_t> t(n, 0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      if ((rows[i] >> j) & 1u) t[j] |= 1u << i;
  return t;
}

struct Contribution {
  uint64_t key;   // x << 32 | z
  double v;
};

// Emits the 2^K X^x Z^z strings of coeff * L_0 L_1 ... L_{K-1} (L_0 leftmost).
void expand(const Encoding& enc, const int* modes, const bool* dagger, int k, double coeff,
            std::vector<Contribution>& out) {
  for (int choice = 0; choice < (1 << k); ++choice) {
    uint32_t x = 0, z = 0;
    double v = coeff;
    for (int m = 0; m < k; ++m) {
      int j = modes[m];
      bool second = (choice >> m) & 1;
      // moving the accumulated Z^z through this string's X^x costs one sign per shared qubit
      if (parity32(z & enc.x[j])) v = -v;
      v *= (dagger[m] || !second) ? 0.5 : -0.5;
      x ^= enc.x[j];
      z ^= enc.zp[j] ^ (second ? enc.ze[j] : 0u);
    }
    out.push_back({((uint64_t)x << 32) | z, v});
  }
}

// Sorts contributions by key and emits one correctly rounded coefficient per key.
void accumulate(std::vector<Contribution>& c, double drop, int n, PauliTerms& out) {
  std::sort(c.begin(), c.end(), [](const Contribution& a, const Contribution& b) {
    return a.key < b.key;
  });
  out = PauliTerms();
  out.n = n;
  ExactSum acc;
  size_t i = 0;
  while (i < c.size()) {
    size_t j = i;
    acc.clear();
    while (j < c.size() && c[j].key == c[i].key) acc.add(c[j++].v);
    double s = acc.round();
    if (s != 0.0 && !(std::fabs(s) < drop)) {
      out.x.push_back((uint32_t)(c[i].key >> 32));
      out.z.push_back((uint32_t)c[i].key);
      out.phase.push_back(0);
      out.coeff.push_back(s);
    }
    i = j;
  }
}

}  // namespace

uint32_t Encoding::encode(uint32_t occupation) const { return apply_rows(beta_rows, occupation); }
uint32_t Encoding::decode(uint32_t qubits) const { return apply_rows(inv_rows, qubits); }

Encoding make_encoding(int mapping, int n) {
  Encoding e;
  e.n = n;
  e.beta_rows.assign(n, 0);
  for (int j = 0; j < n; ++j) {
    if (mapping == GOCP_JW) {
      e.beta_rows[j] = 1u << j;
    } else {
      // Fenwick tree: BK bit j holds the parity of occupations j+1-lowbit(j+1) .. j
      int low = (j + 1) & -(j + 1);
      for (int k = j + 1 - low; k <= j; ++k) e.beta_rows[j] |= 1u << k;
    }
  }
  std::vector<uint32_t> inv = gf2_inverse_rows(e.beta_rows, n);
  e.inv_rows = inv;
  std::vector<uint32_t> inv_t = transpose_rows(inv, n);          // rows of beta^-T
  e.x.resize(n);
  e.zp.resize(n);
  e.ze.resize(n);
  for (int j = 0; j < n; ++j) {
    e.x[j] = apply_rows(e.beta_rows, 1u << j);                  // beta e_j
    e.zp[j] = apply_rows(inv_t, (1u << j) - 1u);                // beta^-T m_j
    e.ze[j] = apply_rows(inv_t, 1u << j);                       // beta^-T e_j
  }
  return e;
}

int build_hamiltonian(const gocp_build_args& a, PauliTerms& out) {
  const int no = a.n_orb, n = 2 * no;
  Encoding enc = make_encoding(a.mapping, n);
  auto drop = [&](double v) { return std::fabs(v) < a.int_drop ? 0.0 : v; };
  std::vector<Contribution> c;
  c.reserve((size_t)no * no * no * no * 4 * 16 / 2 + (size_t)no * no * 8 + 1);
  c.push_back({0, a.e0});
  // one-body: h_pq a+_{p s} a_{q s}
  for (int p = 0; p < no; ++p)
    for (int q = 0; q < no; ++q) {
      double v = drop(a.h[p * no + q]);
      if (v == 0.0) continue;
      for (int s = 0; s < 2; ++s) {
        int modes[2] = {2 * p + s, 2 * q + s};
        bool dag[2] = {true, false};
        expand(enc, modes, dag, 2, v, c);
      }
    }
  // two-body: 1/2 (pq|rs) a+_{p s} a+_{r t} a_{s t} a_{q s}
  for (int p = 0; p < no; ++p)
    for (int q = 0; q < no; ++q)
      for (int r = 0; r < no; ++r)
        for (int s = 0; s < no; ++s) {
          double v = drop(a.g[((size_t)(p * no + q) * no + r) * no + s]);
          if (v == 0.0) continue;
          for (int sg = 0; sg < 2; ++sg)
            for (int tu = 0; tu < 2; ++tu) {
              int modes[4] = {2 * p + sg, 2 * r + tu, 2 * s + tu, 2 * q + sg};
              bool dag[4] = {true, true, false, false};
              expand(enc, modes, dag, 4, 0.5 * v, c);
            }
        }
  accumulate(c, a.term_drop, n, out);
  return GOCP_OK;
}

void build_pool(int n, int n_elec, const Encoding& enc, Pool& out) {
  out = Pool();
  out.off.push_back(0);
  std::vector<Contribution> c;
  PauliTerms t;
  auto emit = [&](const int* fwd, const int* bwd, const bool* dag, int k) {
    c.clear();
    expand(enc, fwd, dag, k, 1.0, c);
    expand(enc, bwd, dag, k, -1.0, c);
    accumulate(c, 0.0, n, t);
    for (size_t i = 0; i < t.size(); ++i) {
      out.x.push_back(t.x[i]);
      out.z.push_back(t.z[i]);
      out.phase.push_back(0);
      out.coeff.push_back(t.coeff[i]);
    }
    out.off.push_back((int64_t)out.x.size());
  };
  // singles: a+_a a_i - a+_i a_a, same spin, ordered by (i, a)
  for (int i = 0; i < n_elec; ++i)
    for (int a = n_elec; a < n; ++a) {
      if ((i & 1) != (a & 1)) continue;
      int fwd[2] = {a, i}, bwd[2] = {i, a};
      bool dag[2] = {true, false};
      emit(fwd, bwd, dag, 2);
    }
  // doubles: a+_a a+_b a_j a_i - h.c., i<j, a<b, S_z conserved, ordered by (i, j, a, b)
  for (int i = 0; i < n_elec; ++i)
    for (int j = i + 1; j < n_elec; ++j)
      for (int a = n_elec; a < n; ++a)
        for (int b = a + 1; b < n; ++b) {
          if ((i & 1) + (j & 1) != (a & 1) + (b & 1)) continue;
          int fwd[4] = {a, b, j, i}, bwd[4] = {i, j, b, a};
          bool dag[4] = {true, true, false, false};
          emit(fwd, bwd, dag, 4);
        }
  out.family.assign(out.size(), -1);
  out.n_families = 0;
}

int canonicalize_terms(const std::vector<uint32_t>& x, const std::vector<uint32_t>& z,
                       const std::vector<uint8_t>& ph, const std::vector<double>& c, double drop,
                       int n, PauliTerms& out) {
  // c i^phase = (+-c) i^(phase mod 2): sum real-phase and imaginary-phase parts separately
  std::vector<Contribution> re, im;
  for (size_t i = 0; i < x.size(); ++i) {
    double v = (ph[i] & 2) ? -c[i] : c[i];
    ((ph[i] & 1) ? im : re).push_back({((uint64_t)x[i] << 32) | z[i], v});
  }
  PauliTerms tr, ti;
  accumulate(re, drop, n, tr);
  accumulate(im, drop, n, ti);
  out = PauliTerms();
  out.n = n;
  size_t a = 0, b = 0;
  while (a < tr.size() || b < ti.size()) {
    uint64_t ka = a < tr.size() ? ((uint64_t)tr.x[a] << 32 | tr.z[a]) : ~0ull;
    uint64_t kb = b < ti.size() ? ((uint64_t)ti.x[b] << 32 | ti.z[b]) : ~0ull;
    if (ka == kb) return fail(GOCP_EINVAL, "a Pauli string has both real and imaginary coefficient parts");
    bool take_a = ka < kb;
    const PauliTerms& src = take_a ? tr : ti;
    size_t k = take_a ? a++ : b++;
    out.x.push_back(src.x[k]);
    out.z.push_back(src.z[k]);
    out.phase.push_back(take_a ? 0 : 1);
    out.coeff.push_back(src.coeff[k]);
  }
  return GOCP_OK;
}

// ------------------------------------------------------------ LUT form

LutForm lut_form(const uint32_t* z, const double* w, int count) {
  LutForm f;
  if (count <= 0) return f;
  f.z0 = z[0];
  // basis of the differences by insertion, each vector reduced against the
  // previous ones (pivot = highest set bit), coordinates tracked alongside
  uint32_t basis[32];
  uint32_t coord_of_basis[32];   // basis[i] expressed in the chosen v's
  int rank = 0;
  std::vector<uint32_t> coords(count, 0);
  for (int t = 0; t < count; ++t) {
    uint32_t r = z[t] ^ f.z0, c = 0;
    for (int i = 0; i < rank; ++i)
      if ((r ^ basis[i]) < r) {
        r ^= basis[i];
        c ^= coord_of_basis[i];
      }
    if (r) {
      if (rank == kMaxLutRank) return LutForm();
      f.v[rank] = r;
      basis[rank] = r;
      coord_of_basis[rank] = 1u << rank;
      c ^= 1u << rank;
      ++rank;
      // keep basis sorted by pivot so that the reduction above stays greedy
      for (int i = rank - 1; i > 0 && basis[i] > basis[i - 1]; --i) {
        std::swap(basis[i], basis[i - 1]);
        std::swap(coord_of_basis[i], coord_of_basis[i - 1]);
      }
    }
    coords[t] = c;
  }
  f.d = rank;
  ExactSum acc;
  for (int sidx = 0; sidx < (1 << rank); ++sidx) {
    acc.clear();
    for (int t = 0; t < count; ++t) acc.add(parity32(coords[t] & (uint32_t)sidx) ? -w[t] : w[t]);
    f.lut[sidx] = acc.round();
  }
  f.ok = true;
  return f;
}

// ------------------------------------------------------------ GOCP

namespace {

struct IntString {
  uint32_t z;
  int64_t re, im;   // 8 * coeff * i^phase as a Gaussian integer
};

bool commutes(uint32_t xa, const std::vector<IntString>& a, uint32_t xb,
              const std::vector<IntString>& b) {
  // [A, B] = sum_{s,t} w_s w_t ((-1)^(z_s.x_b) - (-1)^(z_t.x_a)) X^(xa^xb) Z^(z_s^z_t)
  uint32_t keys[64];
  int64_t sr[64], si[64];
  int nk = 0;
  for (const auto& s : a)
    for (const auto& t : b) {
      int d = (parity32(s.z & xb) ? -1 : 1) - (parity32(t.z & xa) ? -1 : 1);
      if (d == 0) continue;
      uint32_t k = s.z ^ t.z;
      int64_t wr = (s.re * t.re - s.im * t.im) * d;
      int64_t wi = (s.re * t.im + s.im * t.re) * d;
      int f = 0;
      while (f < nk && keys[f] != k) ++f;
      if (f == nk) { keys[nk] = k; sr[nk] = 0; si[nk] = 0; ++nk; }
      sr[f] += wr;
      si[f] += wi;
    }
  for (int f = 0; f < nk; ++f)
    if (sr[f] != 0 || si[f] != 0) return false;
  return true;
}

}  // namespace

int colour_pool(Pool& pool) {
  const int m = pool.size();
  std::vector<std::vector<IntString>> ops(m);
  std::vector<uint32_t> opx(m);
  for (int k = 0; k < m; ++k) {
    int64_t b = pool.off[k], e = pool.off[k + 1];
    if (e - b > 8) return fail(GOCP_EINVAL, "GOCP colouring supports generators of at most 8 strings");
    opx[k] = e > b ? pool.x[b] : 0;
    for (int64_t s = b; s < e; ++s) {
      double w = pool.coeff[s] * 8.0;
      if (w != std::nearbyint(w) || std::fabs(w) > 1e15)
        return fail(GOCP_EINVAL, "GOCP colouring needs generator coefficients that are multiples of 1/8");
      int64_t c = (int64_t)w;
      int ph = pool.phase[s] & 3;
      IntString is{pool.z[s], 0, 0};
      if (ph == 0) is.re = c; else if (ph == 1) is.im = c; else if (ph == 2) is.re = -c; else is.im = -c;
      ops[k].push_back(is);
    }
  }
  // non-commutativity graph as bit rows
  const int words = (m + 63) / 64;
  std::vector<uint64_t> adj((size_t)m * words, 0);
  std::vector<int> degree(m, 0);
  for (int i = 0; i < m; ++i)
    for (int j = i + 1; j < m; ++j)
      if (!commutes(opx[i], ops[i], opx[j], ops[j])) {
        adj[(size_t)i * words + j / 64] |= 1ull << (j % 64);
        adj[(size_t)j * words + i / 64] |= 1ull << (i % 64);
        ++degree[i];
        ++degree[j];
      }
  // Largest-First order (descending degree, pool order within ties)
  std::vector<int> order(m);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return degree[a] > degree[b]; });
  pool.family.assign(m, -1);
  int k_fam = 0;
  std::vector<char> taken;
  for (int v : order) {
    taken.assign(k_fam + 1, 0);
    for (int w = 0; w < words; ++w) {
      uint64_t bits = adj[(size_t)v * words + w];
      while (bits) {
        int u = w * 64 + __builtin_ctzll(bits);
        bits &= bits - 1;
        if (pool.family[u] >= 0) taken[pool.family[u]] = 1;
      }
    }
    int f = 0;
    while (f < k_fam && taken[f]) ++f;   // lowest-index family with no neighbour
    if (f == k_fam) ++k_fam;             // none: open a new family
    pool.family[v] = f;
  }
  pool.n_families = k_fam;
  return GOCP_OK;
}

}  // namespace gocp

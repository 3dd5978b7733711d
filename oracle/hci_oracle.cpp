// Plain CPU oracle for the variational HCI solve (test infrastructure only).
//
// This file is the slow, obviously-correct restatement of what the GPU path
// computes.  It is used by the tests, by __graft_entry__.smoke() and by the
// CPU-baseline leg of bench.py; the product path never links or calls it.
// It shares no code, header, table or constant with the CUDA library.
//
// Conventions (Sec. II of arXiv:1708.07544 states the method; the layout is ours):
//   * determinant = (alpha bits, beta bits), bit p set <=> spatial orbital p occupied;
//   * spin-orbital order: all alpha (0..n-1) then all beta (n..2n-1); the
//     determinant is prod_{alpha occ, ascending} a+ prod_{beta occ, ascending} a+ |0>;
//   * H = sum_pq h_pq sum_s a+_ps a_qs + 1/2 sum_pqrs (pq|rs) sum_st a+_ps a+_rt a_st a_qs + E_core.
//
// Matrix elements follow the textbook Slater-Condon rules (diagonal, single,
// double).  The RDMs are taken from the operator definition, applying
// annihilation/creation operators one at a time with Jordan-Wigner phases.
// Selection (Eq. criteria and the HCI importance function, Sec. II.A)
// enumerates EVERY single and double excitation of every determinant in V
// and keeps D_a not in V with max_i |H_ai c_i| > eps1 (eps1 <= 0: keep all).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <unordered_map>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

struct Key {
  uint64_t a, b;
  bool operator==(const Key& o) const { return a == o.a && b == o.b; }
  bool operator<(const Key& o) const { return a < o.a || (a == o.a && b < o.b); }
};
struct KeyHash {
  size_t operator()(const Key& k) const {
    uint64_t x = k.a * 0x9E3779B97F4A7C15ull ^ (k.b + 0x632BE59BD9B4E019ull + (k.a << 6) + (k.a >> 2));
    x ^= x >> 31; x *= 0xBF58476D1CE4E5B9ull; x ^= x >> 29;
    return (size_t)x;
  }
};

struct Ham {
  int n;
  const double* h;
  const double* eri;
  double ecore;
  double H1(int p, int q) const { return h[p * n + q]; }
  double V(int p, int q, int r, int s) const { return eri[((p * n + q) * n + r) * n + s]; }
};

inline int popc(uint64_t x) { return __builtin_popcountll(x); }
inline bool bit(uint64_t x, int p) { return (x >> p) & 1ull; }

// number of set bits strictly between orbitals p and r
inline int between(uint64_t s, int p, int r) {
  int lo = std::min(p, r), hi = std::max(p, r);
  if (hi - lo <= 1) return 0;
  uint64_t mask = ((hi >= 64 ? ~0ull : ((1ull << hi) - 1ull))) & ~((1ull << (lo + 1)) - 1ull);
  return popc(s & mask);
}
inline double exc_sign(uint64_t s, int p, int r) { return (between(s, p, r) & 1) ? -1.0 : 1.0; }

std::vector<int> occ_list(uint64_t s, int n) {
  std::vector<int> o;
  for (int p = 0; p < n; ++p) if (bit(s, p)) o.push_back(p);
  return o;
}

// <D|H|D>
double diag_element(const Ham& H, uint64_t sa, uint64_t sb) {
  const int n = H.n;
  std::vector<int> oa = occ_list(sa, n), ob = occ_list(sb, n);
  double e = H.ecore;
  for (int p : oa) e += H.H1(p, p);
  for (int p : ob) e += H.H1(p, p);
  // same spin pairs (ordered pairs, halved)
  for (const auto* o : {&oa, &ob}) {
    for (int p : *o) for (int q : *o) if (p != q) e += 0.5 * (H.V(p, p, q, q) - H.V(p, q, q, p));
  }
  for (int p : oa) for (int q : ob) e += H.V(p, p, q, q);
  return e;
}

// <D'|H|D> for D' = a+_r a_p D in spin string `s` (the other spin string is `o`)
double single_element(const Ham& H, uint64_t s, uint64_t o, int p, int r) {
  const int n = H.n;
  double v = H.H1(p, r);
  for (int k = 0; k < n; ++k) {
    if (bit(s, k)) v += H.V(p, r, k, k) - H.V(p, k, k, r);
    if (bit(o, k)) v += H.V(p, r, k, k);
  }
  return exc_sign(s, p, r) * v;
}

// Visit every single and double excitation D_a of D = (sa, sb) with H_aD.
template <class F>
void for_each_excitation(const Ham& H, uint64_t sa, uint64_t sb, F&& f) {
  const int n = H.n;
  for (int spin = 0; spin < 2; ++spin) {
    uint64_t s = spin == 0 ? sa : sb, o = spin == 0 ? sb : sa;
    for (int p = 0; p < n; ++p) {
      if (!bit(s, p)) continue;
      for (int r = 0; r < n; ++r) {
        if (bit(s, r)) continue;
        uint64_t t = s ^ (1ull << p) ^ (1ull << r);
        double v = single_element(H, s, o, p, r);
        if (spin == 0) f(t, sb, v); else f(sa, t, v);
      }
    }
    // same-spin doubles p<q -> r<s
    for (int p = 0; p < n; ++p) {
      if (!bit(s, p)) continue;
      for (int q = p + 1; q < n; ++q) {
        if (!bit(s, q)) continue;
        for (int r = 0; r < n; ++r) {
          if (bit(s, r)) continue;
          for (int w = r + 1; w < n; ++w) {
            if (bit(s, w)) continue;
            double s1 = exc_sign(s, p, r);
            uint64_t t1 = s ^ (1ull << p) ^ (1ull << r);
            double s2 = exc_sign(t1, q, w);
            uint64_t t2 = t1 ^ (1ull << q) ^ (1ull << w);
            double v = s1 * s2 * (H.V(p, r, q, w) - H.V(p, w, q, r));
            if (spin == 0) f(t2, sb, v); else f(sa, t2, v);
          }
        }
      }
    }
  }
  // opposite-spin doubles: alpha p->r, beta q->s
  for (int p = 0; p < n; ++p) {
    if (!bit(sa, p)) continue;
    for (int r = 0; r < n; ++r) {
      if (bit(sa, r)) continue;
      double s1 = exc_sign(sa, p, r);
      uint64_t ta = sa ^ (1ull << p) ^ (1ull << r);
      for (int q = 0; q < n; ++q) {
        if (!bit(sb, q)) continue;
        for (int w = 0; w < n; ++w) {
          if (bit(sb, w)) continue;
          double s2 = exc_sign(sb, q, w);
          uint64_t tb = sb ^ (1ull << q) ^ (1ull << w);
          f(ta, tb, s1 * s2 * H.V(p, r, q, w));
        }
      }
    }
  }
}

struct Index {
  std::unordered_map<Key, int64_t, KeyHash> m;
  Index(const uint64_t* keys, int64_t nV) {
    m.reserve((size_t)nV * 2 + 1);
    for (int64_t i = 0; i < nV; ++i) m.emplace(Key{keys[2 * i], keys[2 * i + 1]}, i);
  }
  int64_t find(uint64_t a, uint64_t b) const {
    auto it = m.find(Key{a, b});
    return it == m.end() ? -1 : it->second;
  }
};

struct Csr {
  std::vector<int64_t> rowptr;
  std::vector<int64_t> col;
  std::vector<double> val;
};

struct Selection {
  std::vector<uint64_t> keys;  // (a, b) pairs, sorted
  std::vector<double> f;       // max_i |H_ai c_i| of each listed determinant
};

// Jordan-Wigner phase of acting on spin-orbital m of a determinant: (-1)^(occupied modes below m)
inline int mode_of(int n, int p, int spin) { return spin * n + p; }
inline bool occ_mode(uint64_t sa, uint64_t sb, int n, int m) { return m < n ? bit(sa, m) : bit(sb, m - n); }
inline int below(uint64_t sa, uint64_t sb, int n, int m) {
  if (m < n) return popc(sa & ((1ull << m) - 1ull));
  int mb = m - n;
  return popc(sa) + popc(sb & ((1ull << mb) - 1ull));
}
inline void flip(uint64_t& sa, uint64_t& sb, int n, int m) {
  if (m < n) sa ^= (1ull << m); else sb ^= (1ull << (m - n));
}
// apply a_m (create=false) or a+_m (create=true); returns false if result is zero
inline bool apply_op(uint64_t& sa, uint64_t& sb, int n, int m, bool create, double& sign) {
  bool o = occ_mode(sa, sb, n, m);
  if (create == o) return false;
  if (below(sa, sb, n, m) & 1) sign = -sign;
  flip(sa, sb, n, m);
  return true;
}

}  // namespace

extern "C" {

// Diagonal elements H_ii for every determinant.
void orc_diag(int n, const double* h, const double* eri, double ecore, const uint64_t* keys,
              int64_t nV, double* out) {
  Ham H{n, h, eri, ecore};
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t i = 0; i < nV; ++i) out[i] = diag_element(H, keys[2 * i], keys[2 * i + 1]);
}

// Full Hamiltonian on V in CSR (rows i, columns j, <D_i|H|D_j>), diagonal included.
void* orc_hamiltonian(int n, const double* h, const double* eri, double ecore, const uint64_t* keys,
                      int64_t nV) {
  Ham H{n, h, eri, ecore};
  Index idx(keys, nV);
  std::vector<std::vector<std::pair<int64_t, double>>> rows((size_t)nV);
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t j = 0; j < nV; ++j) {
    auto& row = rows[(size_t)j];
    row.emplace_back(j, diag_element(H, keys[2 * j], keys[2 * j + 1]));
    // <D_a|H|D_j> for every excitation a of j; by symmetry H_ja = H_aj
    for_each_excitation(H, keys[2 * j], keys[2 * j + 1], [&](uint64_t a, uint64_t b, double v) {
      int64_t i = idx.find(a, b);
      if (i >= 0) row.emplace_back(i, v);
    });
    std::sort(row.begin(), row.end());
  }
  Csr* m = new Csr;
  m->rowptr.resize((size_t)nV + 1, 0);
  for (int64_t i = 0; i < nV; ++i) m->rowptr[i + 1] = m->rowptr[i] + (int64_t)rows[i].size();
  m->col.resize((size_t)m->rowptr[nV]);
  m->val.resize((size_t)m->rowptr[nV]);
  for (int64_t i = 0; i < nV; ++i) {
    int64_t o = m->rowptr[i];
    for (size_t k = 0; k < rows[i].size(); ++k) {
      m->col[o + k] = rows[i][k].first;
      m->val[o + k] = rows[i][k].second;
    }
  }
  return m;
}
int64_t orc_csr_nnz(void* p) { return ((Csr*)p)->rowptr.back(); }
void orc_csr_copy(void* p, int64_t* rowptr, int64_t* col, double* val) {
  Csr* m = (Csr*)p;
  std::memcpy(rowptr, m->rowptr.data(), m->rowptr.size() * sizeof(int64_t));
  std::memcpy(col, m->col.data(), m->col.size() * sizeof(int64_t));
  std::memcpy(val, m->val.data(), m->val.size() * sizeof(double));
}
void orc_csr_free(void* p) { delete (Csr*)p; }

// sigma_i = sum_j H_ij c_j for the listed rows only (enumeration + lookup).
void orc_sigma_rows(int n, const double* h, const double* eri, double ecore, const uint64_t* keys,
                    int64_t nV, const double* c, const int64_t* rows, int64_t nrows, double* out) {
  Ham H{n, h, eri, ecore};
  Index idx(keys, nV);
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t t = 0; t < nrows; ++t) {
    int64_t i = rows[t];
    double acc = diag_element(H, keys[2 * i], keys[2 * i + 1]) * c[i];
    for_each_excitation(H, keys[2 * i], keys[2 * i + 1], [&](uint64_t a, uint64_t b, double v) {
      int64_t j = idx.find(a, b);
      if (j >= 0) acc += v * c[j];
    });
    out[t] = acc;
  }
}

// Selection step: every single/double D_a of every D_i in V with D_a not in V.
// Returns the determinants whose f(D_a) = max_i |H_ai c_i| exceeds
// list_floor (the caller passes eps1*(1-band) to also see near-misses).
// With all_excitations != 0 every excitation is listed (f still reported).
void* orc_select(int n, const double* h, const double* eri, const uint64_t* keys, const double* c,
                 int64_t nV, double list_floor, int all_excitations, const int64_t* sources,
                 int64_t nsources) {
  Ham H{n, h, eri, 0.0};
  Index idx(keys, nV);
  std::unordered_map<Key, double, KeyHash> best;
  int64_t count = sources ? nsources : nV;
#ifdef _OPENMP
  int nt = omp_get_max_threads();
#else
  int nt = 1;
#endif
  std::vector<std::unordered_map<Key, double, KeyHash>> part((size_t)nt);
#pragma omp parallel
  {
#ifdef _OPENMP
    int tid = omp_get_thread_num();
#else
    int tid = 0;
#endif
    auto& mine = part[(size_t)tid];
#pragma omp for schedule(dynamic, 8)
    for (int64_t t = 0; t < count; ++t) {
      int64_t i = sources ? sources[t] : t;
      double ci = std::fabs(c[i]);
      for_each_excitation(H, keys[2 * i], keys[2 * i + 1], [&](uint64_t a, uint64_t b, double v) {
        double fv = std::fabs(v) * ci;
        if (!all_excitations && !(fv > list_floor)) return;
        if (idx.find(a, b) >= 0) return;
        Key k{a, b};
        auto it = mine.find(k);
        if (it == mine.end()) mine.emplace(k, fv);
        else if (fv > it->second) it->second = fv;
      });
    }
  }
  for (auto& m : part)
    for (auto& kv : m) {
      auto it = best.find(kv.first);
      if (it == best.end()) best.emplace(kv.first, kv.second);
      else if (kv.second > it->second) it->second = kv.second;
    }
  std::vector<std::pair<Key, double>> v(best.begin(), best.end());
  std::sort(v.begin(), v.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
  Selection* s = new Selection;
  s->keys.reserve(v.size() * 2);
  s->f.reserve(v.size());
  for (auto& kv : v) {
    s->keys.push_back(kv.first.a);
    s->keys.push_back(kv.first.b);
    s->f.push_back(kv.second);
  }
  return s;
}
// Second-order Epstein-Nesbet correction with screening (Sec. II.B,
// Eq. pt_hci):  E2 = sum over D_a not in V of (sum'_i H_ai c_i)^2 / (e0 - H_aa),
// where the screened sum keeps the terms with |H_ai c_i| > eps2 and D_a
// belongs to C(eps2) when at least one term is kept.  Every single and double
// of every D_i is enumerated.  Each thread owns the targets of one hash
// class and adds their terms in ascending source order; the contributions
// are summed in ascending key order, so the result does not depend on the
// number of threads.
void orc_pt2(int n, const double* h, const double* eri, double ecore, const uint64_t* keys, const double* c,
             int64_t nV, double eps2, double e0, double* e2, int64_t* n_ext) {
  Ham H{n, h, eri, ecore};
  Index idx(keys, nV);
#ifdef _OPENMP
  int nt = omp_get_max_threads();
#else
  int nt = 1;
#endif
  std::vector<std::vector<std::pair<Key, double>>> contrib((size_t)nt);
#pragma omp parallel num_threads(nt)
  {
#ifdef _OPENMP
    int tid = omp_get_thread_num();
#else
    int tid = 0;
#endif
    std::unordered_map<Key, double, KeyHash> num;
    KeyHash kh;
    for (int64_t i = 0; i < nV; ++i) {
      const double ci = c[i];
      for_each_excitation(H, keys[2 * i], keys[2 * i + 1], [&](uint64_t a, uint64_t b, double v) {
        const Key k{a, b};
        if ((int)(kh(k) % (size_t)nt) != tid) return;
        const double t = v * ci;
        if (!(std::fabs(t) > eps2)) return;
        if (idx.find(a, b) >= 0) return;
        num[k] += t;
      });
    }
    auto& out = contrib[(size_t)tid];
    out.reserve(num.size());
    for (auto& kv : num) {
      const double haa = diag_element(H, kv.first.a, kv.first.b);
      out.emplace_back(kv.first, kv.second * kv.second / (e0 - haa));
    }
  }
  std::vector<std::pair<Key, double>> all;
  for (auto& v : contrib) all.insert(all.end(), v.begin(), v.end());
  std::sort(all.begin(), all.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
  double sum = 0.0;
  for (auto& kv : all) sum += kv.second;
  *e2 = sum;
  *n_ext = (int64_t)all.size();
}

// One sample of the stochastic second-order correction (Sec. II.B, the
// unbiased multinomial estimator of the cited semistochastic HCI work,
// Eq. semistoc).  The sample is n_draws determinants drawn from V with
// replacement, D_j with probability p_j; the distinct ones are given with
// f_j = w_j / p_j (w_j = times drawn).  For every target D_a outside V, over
// the sampled pairs kept by a screen (|H_aj c_j| > eps), with x_j = H_aj c_j:
//   S = sum_j f_j x_j,  T = sum_j (f_j x_j)^2,  U = sum_j f_j x_j^2,
//   e_a = (S^2 - T + (N_d - 1) U) / (N_d (N_d - 1) (e0 - H_aa)),
// which is the estimator's [(sum_j w_j x_j / p_j)^2 + sum_j (w_j (N_d - 1) /
// p_j - w_j^2 / p_j^2) x_j^2] / (N_d (N_d - 1) (e0 - H_aa)) with its terms
// grouped so that a target reached from one sampled determinant has
// S^2 - T = 0 exactly.  Its expectation over the draws is E2 with the same
// screen.  out[0] uses eps2, out[1] eps2_det (>= eps2).  Targets are summed
// in ascending key order.
void orc_pt2_sampled(int n, const double* h, const double* eri, double ecore, const uint64_t* keys, int64_t nV,
                     const uint64_t* src_keys, const double* src_c, const double* src_f, int64_t nsrc,
                     int64_t n_draws, double eps2, double eps2_det, double e0, double* out) {
  Ham H{n, h, eri, ecore};
  Index idx(keys, nV);
  struct Acc { double s[2], t[2], u[2]; };
  std::map<Key, Acc> acc;
  for (int64_t j = 0; j < nsrc; ++j) {
    const double cj = src_c[j], fj = src_f[j];
    for_each_excitation(H, src_keys[2 * j], src_keys[2 * j + 1], [&](uint64_t a, uint64_t b, double v) {
      const double x = v * cj;
      if (!(std::fabs(x) > eps2)) return;
      if (idx.find(a, b) >= 0) return;
      Acc& r = acc.try_emplace(Key{a, b}, Acc{{0, 0}, {0, 0}, {0, 0}}).first->second;
      for (int k = 0; k < 2; ++k) {
        if (k == 1 && !(std::fabs(x) > eps2_det)) break;
        r.s[k] += fj * x;
        r.t[k] += (fj * x) * (fj * x);
        r.u[k] += fj * x * x;
      }
    });
  }
  const double nd = (double)n_draws;
  double e[2] = {0.0, 0.0};
  for (auto& kv : acc) {
    const double den = nd * (nd - 1.0) * (e0 - diag_element(H, kv.first.a, kv.first.b));
    for (int k = 0; k < 2; ++k) {
      const Acc& r = kv.second;
      e[k] += (r.s[k] * r.s[k] - r.t[k] + (nd - 1.0) * r.u[k]) / den;
    }
  }
  out[0] = e[0];
  out[1] = e[1];
}

// Density matrices of the perturbative correction (Sec. V, Computational
// Details), in the spin-summed order of orc_rdm12:
//   dd:  sum over D_a in C(eps2) of d_a^2 <D_a| op |D_a>
//   dc:  sum over the screened pairs (D_i in V, D_a in C(eps2)) of
//        c_i d_a <D_i| op |D_a>
// with d_a = (sum'_i H_ai c_i) / (e0 - H_aa), the same screened sum as
// orc_pt2 (a pair is kept when |H_ai c_i| > eps2).  Every operator string
// is applied to the ket determinant and the result compared with the bra.
static void pair_rdm(int n, uint64_t ka, uint64_t kb, uint64_t ba, uint64_t bb, double w, double* g1, double* g2) {
  const int M = 2 * n;
  for (int s = 0; s < 2; ++s)
    for (int q = 0; q < n; ++q)
      for (int p = 0; p < n; ++p) {
        uint64_t a = ka, b = kb;
        double sg = 1.0;
        if (!apply_op(a, b, n, mode_of(n, q, s), false, sg)) continue;
        if (!apply_op(a, b, n, mode_of(n, p, s), true, sg)) continue;
        if (a == ba && b == bb) g1[(size_t)p * n + q] += w * sg;
      }
  for (int mq = 0; mq < M; ++mq) {
    uint64_t a1 = ka, b1 = kb;
    double sg1 = 1.0;
    if (!apply_op(a1, b1, n, mq, false, sg1)) continue;
    for (int ms = 0; ms < M; ++ms) {
      uint64_t a2 = a1, b2 = b1;
      double sg2 = sg1;
      if (!apply_op(a2, b2, n, ms, false, sg2)) continue;
      const int spinq = mq / n, spins = ms / n;
      for (int mr = spins * n; mr < spins * n + n; ++mr) {
        uint64_t a3 = a2, b3 = b2;
        double sg3 = sg2;
        if (!apply_op(a3, b3, n, mr, true, sg3)) continue;
        for (int mp = spinq * n; mp < spinq * n + n; ++mp) {
          uint64_t a4 = a3, b4 = b3;
          double sg4 = sg3;
          if (!apply_op(a4, b4, n, mp, true, sg4)) continue;
          if (a4 != ba || b4 != bb) continue;
          const int p = mp % n, q = mq % n, r = mr % n, s = ms % n;
          g2[(((size_t)p * n + q) * n + r) * n + s] += w * sg4;
        }
      }
    }
  }
}

void orc_pt2_rdm(int n, const double* h, const double* eri, double ecore, const uint64_t* keys, const double* c,
                 int64_t nV, double eps2, double e0, double* rdm1_dd, double* rdm2_dd, double* rdm1_dc,
                 double* rdm2_dc) {
  Ham H{n, h, eri, ecore};
  Index idx(keys, nV);
  std::unordered_map<Key, double, KeyHash> num;
  std::vector<std::pair<int64_t, Key>> pairs;
  for (int64_t i = 0; i < nV; ++i) {
    const double ci = c[i];
    for_each_excitation(H, keys[2 * i], keys[2 * i + 1], [&](uint64_t a, uint64_t b, double v) {
      const double t = v * ci;
      if (!(std::fabs(t) > eps2)) return;
      if (idx.find(a, b) >= 0) return;
      const Key k{a, b};
      num[k] += t;
      pairs.emplace_back(i, k);
    });
  }
  std::unordered_map<Key, double, KeyHash> d;
  for (auto& kv : num) d[kv.first] = kv.second / (e0 - diag_element(H, kv.first.a, kv.first.b));
  const size_t n2 = (size_t)n * n, n4 = n2 * n2;
  std::fill(rdm1_dd, rdm1_dd + n2, 0.0);
  std::fill(rdm2_dd, rdm2_dd + n4, 0.0);
  std::fill(rdm1_dc, rdm1_dc + n2, 0.0);
  std::fill(rdm2_dc, rdm2_dc + n4, 0.0);
  for (auto& kv : d) pair_rdm(n, kv.first.a, kv.first.b, kv.first.a, kv.first.b, kv.second * kv.second, rdm1_dd, rdm2_dd);
  for (auto& pr : pairs) {
    const int64_t i = pr.first;
    const Key& k = pr.second;
    pair_rdm(n, k.a, k.b, keys[2 * i], keys[2 * i + 1], c[i] * d[k], rdm1_dc, rdm2_dc);
  }
}

int64_t orc_sel_count(void* p) { return (int64_t)((Selection*)p)->f.size(); }
void orc_sel_copy(void* p, uint64_t* keys, double* f) {
  Selection* s = (Selection*)p;
  std::memcpy(keys, s->keys.data(), s->keys.size() * sizeof(uint64_t));
  std::memcpy(f, s->f.data(), s->f.size() * sizeof(double));
}
void orc_sel_free(void* p) { delete (Selection*)p; }

// Spin-summed RDMs from the operator definition (Sec. IV):
//   rdm1[p,q]      = sum_s <a+_ps a_qs>
//   rdm2[p,q,r,s]  = sum_st <a+_ps a+_rt a_st a_qs>
// computed as sum_j c_j sum_ops <D_i| op |D_j> c_i with D_i looked up in V.
void orc_rdm12(int n, const uint64_t* keys, int64_t nV, const double* c, double* rdm1, double* rdm2) {
  Index idx(keys, nV);
  const int M = 2 * n;
  const size_t n2 = (size_t)n * n, n4 = n2 * n2;
#ifdef _OPENMP
  int nt = omp_get_max_threads();
#else
  int nt = 1;
#endif
  std::vector<std::vector<double>> r1((size_t)nt, std::vector<double>(n2, 0.0));
  std::vector<std::vector<double>> r2((size_t)nt, std::vector<double>(n4, 0.0));
#pragma omp parallel
  {
#ifdef _OPENMP
    int tid = omp_get_thread_num();
#else
    int tid = 0;
#endif
    auto& g1 = r1[(size_t)tid];
    auto& g2 = r2[(size_t)tid];
#pragma omp for schedule(dynamic, 8)
    for (int64_t j = 0; j < nV; ++j) {
      const uint64_t a0 = keys[2 * j], b0 = keys[2 * j + 1];
      const double cj = c[j];
      if (cj == 0.0) continue;
      // one-body: a+_{p s} a_{q s}
      for (int s = 0; s < 2; ++s)
        for (int q = 0; q < n; ++q)
          for (int p = 0; p < n; ++p) {
            uint64_t a = a0, b = b0;
            double sg = 1.0;
            if (!apply_op(a, b, n, mode_of(n, q, s), false, sg)) continue;
            if (!apply_op(a, b, n, mode_of(n, p, s), true, sg)) continue;
            int64_t i = idx.find(a, b);
            if (i >= 0) g1[(size_t)p * n + q] += c[i] * cj * sg;
          }
      // two-body: a+_{P} a+_{R} a_{S} a_{Q} with P=(p,s1) Q=(q,s1) R=(r,s2) S=(s,s2)
      for (int mq = 0; mq < M; ++mq) {
        uint64_t a1 = a0, b1 = b0;
        double sg1 = 1.0;
        if (!apply_op(a1, b1, n, mq, false, sg1)) continue;
        for (int ms = 0; ms < M; ++ms) {
          uint64_t a2 = a1, b2 = b1;
          double sg2 = sg1;
          if (!apply_op(a2, b2, n, ms, false, sg2)) continue;
          int spinq = mq / n, spins = ms / n;
          for (int mr = spins * n; mr < spins * n + n; ++mr) {
            uint64_t a3 = a2, b3 = b2;
            double sg3 = sg2;
            if (!apply_op(a3, b3, n, mr, true, sg3)) continue;
            for (int mp = spinq * n; mp < spinq * n + n; ++mp) {
              uint64_t a4 = a3, b4 = b3;
              double sg4 = sg3;
              if (!apply_op(a4, b4, n, mp, true, sg4)) continue;
              int64_t i = idx.find(a4, b4);
              if (i < 0) continue;
              int p = mp % n, q = mq % n, r = mr % n, s = ms % n;
              g2[(((size_t)p * n + q) * n + r) * n + s] += c[i] * cj * sg4;
            }
          }
        }
      }
    }
  }
  for (size_t k = 0; k < n2; ++k) {
    double acc = 0.0;
    for (int t = 0; t < nt; ++t) acc += r1[(size_t)t][k];
    rdm1[k] = acc;
  }
  for (size_t k = 0; k < n4; ++k) {
    double acc = 0.0;
    for (int t = 0; t < nt; ++t) acc += r2[(size_t)t][k];
    rdm2[k] = acc;
  }
}

int orc_num_threads() {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

}  // extern "C"

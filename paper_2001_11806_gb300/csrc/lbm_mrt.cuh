// Compile-time MRT moment basis (Sec. III-A "Moment Space", Eq. mrt).
//
// Built at compile time in exact int64 rational arithmetic, following the
// paper's automatic procedure:
//   1. candidate moments are monomials c_x^a c_y^b c_z^c with exponents in
//      {0, 1, 2} (higher powers alias lower ones because c is in {-1,0,1});
//   2. monomials whose row M_kq = P_k(c_q) is all zero are dropped (8 of 27
//      for D3Q19);
//   3. candidates are sorted by order, then lexicographically;
//   4. the diagonal second-order monomials are split into shear differences
//      (x^2 - y^2, x^2 - z^2) and the bulk sum (x^2 + y^2 + z^2); mixed
//      second-order monomials are shear moments;
//   5. Gram-Schmidt with the lattice-weighted scalar product
//      <a, b> = sum_q w_q a_q b_q, applied to the rows, each result scaled to
//      primitive integers.
// Relaxation groups: order < 2 conserved (rate 0), shear, bulk, then one rate
// per order >= 3 (the MRT example of Sec. III-C).
// Because the rows are w-orthogonal, M^-1 = W M^T D^-1 with
// D_k = sum_q w_q M_kq^2, so the collision needs only the integer rows.
#pragma once
#include "lbm_lattice.cuh"

namespace lbm {
namespace mrt {

constexpr long long cgcd(long long a, long long b) {
  a = a < 0 ? -a : a;
  b = b < 0 ? -b : b;
  while (b != 0) { long long t = a % b; a = b; b = t; }
  return a;
}

struct Rat {
  long long n = 0, d = 1;
  constexpr Rat() = default;
  constexpr Rat(long long nn, long long dd = 1) : n(nn), d(dd) {
    if (d < 0) { n = -n; d = -d; }
    long long g = cgcd(n, d);
    if (g > 1) { n /= g; d /= g; }
  }
};
constexpr Rat operator+(Rat a, Rat b) { return Rat(a.n * b.d + b.n * a.d, a.d * b.d); }
constexpr Rat operator-(Rat a, Rat b) { return Rat(a.n * b.d - b.n * a.d, a.d * b.d); }
constexpr Rat operator*(Rat a, Rat b) { return Rat(a.n * b.n, a.d * b.d); }
constexpr Rat operator/(Rat a, Rat b) { return Rat(a.n * b.d, a.d * b.n); }

enum Kind : int { CONSERVED = 0, SHEAR = 1, BULK = 2, HIGHER = 3 };

template <class L>
struct Basis {
  static constexpr int Q = L::Q;
  int M[Q][Q] = {};    // row k, column q: primitive integer moment rows
  int kind[Q] = {};
  int order[Q] = {};
  int group[Q] = {};   // index into the rate array: -1 conserved, 0 shear, 1 bulk, order-1 otherwise
  double invD[Q] = {}; // 1 / sum_q w_q M_kq^2
};

template <class L>
constexpr int mono_value(int q, int a, int b, int c) {
  int v = 1;
  for (int i = 0; i < a; ++i) v *= L::cx(q);
  for (int i = 0; i < b; ++i) v *= L::cy(q);
  for (int i = 0; i < c; ++i) v *= L::cz(q);
  return v;
}

template <class L>
constexpr Basis<L> build() {
  constexpr int Q = L::Q;
  Basis<L> out{};
  // steps 1-2: candidate exponents with a non-zero row
  int ex[27][3] = {};
  int n = 0;
  const int cmax = (L::D == 3) ? 3 : 1;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      for (int c = 0; c < cmax; ++c) {
        bool nz = false;
        for (int q = 0; q < Q; ++q) nz = nz || (mono_value<L>(q, a, b, c) != 0);
        if (nz) { ex[n][0] = a; ex[n][1] = b; ex[n][2] = c; ++n; }
      }
  // step 3: sort by order, then lexicographically (higher x power first, ...)
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) {
      int oi = ex[i][0] + ex[i][1] + ex[i][2], oj = ex[j][0] + ex[j][1] + ex[j][2];
      bool swap = oj < oi;
      if (oj == oi) {
        for (int k = 0; k < 3; ++k) {
          if (ex[j][k] != ex[i][k]) { swap = ex[j][k] > ex[i][k]; break; }
        }
      }
      if (swap)
        for (int k = 0; k < 3; ++k) { int t = ex[i][k]; ex[i][k] = ex[j][k]; ex[j][k] = t; }
    }
  // step 4: candidate rows with the shear/bulk split of the order-2 block
  long long rows[27][27] = {};
  int kind[27] = {}, ord[27] = {};
  int r = 0;
  int diag[3] = {-1, -1, -1};
  for (int i = 0; i < n; ++i) {
    int o = ex[i][0] + ex[i][1] + ex[i][2];
    for (int a = 0; a < L::D; ++a)
      if (o == 2 && ex[i][a] == 2) diag[a] = i;
  }
  for (int i = 0; i < n; ++i) {
    int o = ex[i][0] + ex[i][1] + ex[i][2];
    if (o == 2) {
      bool is_diag = false;
      for (int a = 0; a < L::D; ++a) is_diag = is_diag || (diag[a] == i);
      if (is_diag && i == diag[0]) {
        // shear differences x^2 - y^2 (, x^2 - z^2)
        for (int a = 1; a < L::D; ++a) {
          for (int q = 0; q < Q; ++q)
            rows[r][q] = mono_value<L>(q, ex[diag[0]][0], ex[diag[0]][1], ex[diag[0]][2]) -
                         mono_value<L>(q, ex[diag[a]][0], ex[diag[a]][1], ex[diag[a]][2]);
          kind[r] = SHEAR; ord[r] = 2; ++r;
        }
      } else if (!is_diag) {
        for (int q = 0; q < Q; ++q) rows[r][q] = mono_value<L>(q, ex[i][0], ex[i][1], ex[i][2]);
        kind[r] = SHEAR; ord[r] = 2; ++r;
      }
      // the bulk row follows the last order-2 candidate
      bool last2 = (i + 1 == n) || (ex[i + 1][0] + ex[i + 1][1] + ex[i + 1][2] != 2);
      if (last2) {
        for (int q = 0; q < Q; ++q) {
          long long s = 0;
          for (int a = 0; a < L::D; ++a)
            s += mono_value<L>(q, ex[diag[a]][0], ex[diag[a]][1], ex[diag[a]][2]);
          rows[r][q] = s;
        }
        kind[r] = BULK; ord[r] = 2; ++r;
      }
    } else {
      for (int q = 0; q < Q; ++q) rows[r][q] = mono_value<L>(q, ex[i][0], ex[i][1], ex[i][2]);
      kind[r] = (o < 2) ? CONSERVED : HIGHER;
      ord[r] = o;
      ++r;
    }
  }
  // step 5: weighted Gram-Schmidt on the rows, integer weights w_num / w_den
  long long done[27][27] = {};
  for (int k = 0; k < r; ++k) {
    Rat v[27] = {};
    for (int q = 0; q < Q; ++q) v[q] = Rat(rows[k][q]);
    for (int j = 0; j < k; ++j) {
      long long num = 0, den = 0;
      for (int q = 0; q < Q; ++q) {
        num += L::w_num(q) * rows[k][q] * done[j][q];
        den += L::w_num(q) * done[j][q] * done[j][q];
      }
      if (num != 0) {
        Rat coef(num, den);
        for (int q = 0; q < Q; ++q) v[q] = v[q] - coef * Rat(done[j][q]);
      }
    }
    long long l = 1;
    for (int q = 0; q < Q; ++q) l = l / cgcd(l, v[q].d) * v[q].d;
    long long g = 0;
    for (int q = 0; q < Q; ++q) g = cgcd(g, v[q].n * (l / v[q].d));
    for (int q = 0; q < Q; ++q) done[k][q] = v[q].n * (l / v[q].d) / g;
  }
  for (int k = 0; k < Q; ++k) {
    long long dd = 0;
    for (int q = 0; q < Q; ++q) {
      out.M[k][q] = (int)done[k][q];
      dd += L::w_num(q) * done[k][q] * done[k][q];
    }
    out.invD[k] = (double)L::w_den / (double)dd;
    out.kind[k] = kind[k];
    out.order[k] = ord[k];
    out.group[k] = kind[k] == CONSERVED ? -1 : (kind[k] == SHEAR ? 0 : (kind[k] == BULK ? 1 : ord[k] - 1));
  }
  return out;
}

template <class L>
struct Table {
  static constexpr Basis<L> B = build<L>();
};

}  // namespace mrt
}  // namespace lbm

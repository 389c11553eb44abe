// Homogenisation rules of section 2 -- Voigt (eq. 3), Reuss (eq. 4) and the 2-layer laminate
// (eqs. 5-a, 5-b) -- on full nc x nc Mandel matrices, templated on the scalar type so that the
// filter build evaluates them in double and the backward pass differentiates them in forward mode
// with the dual numbers below.
#pragma once

#include <cmath>

#include "hom_common.cuh"

namespace hom {

// Forward-mode dual number v + d eps (eps^2 = 0).
struct Dual {
  double v, d;
};
HOM_HD Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
HOM_HD Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
HOM_HD Dual operator-(Dual a) { return {-a.v, -a.d}; }
HOM_HD Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.v * b.d + a.d * b.v}; }
HOM_HD Dual operator/(Dual a, Dual b) { return {a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)}; }
HOM_HD Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
HOM_HD Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }
HOM_HD Dual& operator*=(Dual& a, Dual b) { a = a * b; return a; }
HOM_HD Dual operator*(double a, Dual b) { return {a * b.v, a * b.d}; }
HOM_HD Dual operator*(Dual a, double b) { return {a.v * b, a.d * b}; }

template <typename S> HOM_HD S scal(double x);
template <> HOM_HD double scal<double>(double x) { return x; }
template <> HOM_HD Dual scal<Dual>(double x) { return {x, 0.0}; }
HOM_HD double mag(double x) { return x < 0 ? -x : x; }
HOM_HD double mag(Dual x) { return x.v < 0 ? -x.v : x.v; }

// In-place inverse of an m x m matrix (row-major, m <= 6) by Gauss-Jordan with partial pivoting.
// Returns false if a pivot vanishes.
template <typename S>
HOM_HD bool inv_small_t(S* A, int m) {
  S Ainv[36];
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) Ainv[i * m + j] = scal<S>((i == j) ? 1.0 : 0.0);
  for (int c = 0; c < m; ++c) {
    int piv = c;
    double best = mag(A[c * m + c]);
    for (int r = c + 1; r < m; ++r) {
      const double v = mag(A[r * m + c]);
      if (v > best) { best = v; piv = r; }
    }
    if (!(best > 0.0)) return false;
    if (piv != c) {
      for (int j = 0; j < m; ++j) {
        S t = A[c * m + j]; A[c * m + j] = A[piv * m + j]; A[piv * m + j] = t;
        t = Ainv[c * m + j]; Ainv[c * m + j] = Ainv[piv * m + j]; Ainv[piv * m + j] = t;
      }
    }
    const S d = scal<S>(1.0) / A[c * m + c];
    for (int j = 0; j < m; ++j) { A[c * m + j] *= d; Ainv[c * m + j] *= d; }
    for (int r = 0; r < m; ++r) {
      if (r == c) continue;
      const S f = A[r * m + c];
      for (int j = 0; j < m; ++j) { A[r * m + j] -= f * A[c * m + j]; Ainv[r * m + j] -= f * Ainv[c * m + j]; }
    }
  }
  for (int i = 0; i < m * m; ++i) A[i] = Ainv[i];
  return true;
}

// C = A * B (m x k) * (k x p), row-major; either factor may be double.
template <typename SA, typename SB, typename SC>
HOM_HD void matmul_t(const SA* A, const SB* B, SC* C, int m, int k, int p) {
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < p; ++j) {
      SC s = scal<SC>(0.0);
      for (int t = 0; t < k; ++t) s += A[i * k + t] * B[t * p + j];
      C[i * p + j] = s;
    }
}
// Full isotropic Mandel stiffness (plane strain in 2D) of Lame constants (lam, mu).
template <typename S>
HOM_HD void iso_full_t(S lam, S mu, int dim, S* C) {
  const int nc = nc_of(dim);
  for (int i = 0; i < nc * nc; ++i) C[i] = scal<S>(0.0);
  for (int i = 0; i < nc; ++i) C[i * nc + i] = scal<S>(2.0) * mu;
  for (int i = 0; i < dim; ++i)
    for (int j = 0; j < dim; ++j) C[i * nc + j] += lam;
}

// Mandel rotation Q (eps' = Q eps) for the orthonormal rows R (local axes).
HOM_HD void mandel_rotation(const double* R, int dim, double* Q) {
  const int nc = nc_of(dim);
  const double s2 = 1.4142135623730950488;
  for (int I = 0; I < nc; ++I) {
    int i, j;
    mandel_pair(dim, I, i, j);
    const double wI = (i == j) ? 1.0 : s2;
    for (int J = 0; J < nc; ++J) {
      int p, q;
      mandel_pair(dim, J, p, q);
      const double wJ = (p == q) ? 1.0 : s2;
      double v = R[i * dim + p] * R[j * dim + q];
      if (p != q) v += R[i * dim + q] * R[j * dim + p];
      Q[I * nc + J] = wI / wJ * v;
    }
  }
}

// Orthonormal rows (t1[, t2], n) of the interface frame: the normal is the last local axis.
HOM_HD void interface_frame(const double* nrm, int dim, double* R) {
  if (dim == 2) {
    R[0] = nrm[1]; R[1] = -nrm[0];
    R[2] = nrm[0]; R[3] = nrm[1];
    return;
  }
  int m = 0;
  double am = nrm[0] < 0 ? -nrm[0] : nrm[0];
  for (int k = 1; k < 3; ++k) {
    const double a = nrm[k] < 0 ? -nrm[k] : nrm[k];
    if (a < am) { am = a; m = k; }
  }
  double e[3] = {0, 0, 0};
  e[m] = 1.0;
  double t1[3] = {nrm[1] * e[2] - nrm[2] * e[1], nrm[2] * e[0] - nrm[0] * e[2], nrm[0] * e[1] - nrm[1] * e[0]};
  const double l = sqrt(t1[0] * t1[0] + t1[1] * t1[1] + t1[2] * t1[2]);
  for (int k = 0; k < 3; ++k) t1[k] /= l;
  const double t2[3] = {nrm[1] * t1[2] - nrm[2] * t1[1], nrm[2] * t1[0] - nrm[0] * t1[2],
                        nrm[0] * t1[1] - nrm[1] * t1[0]};
  for (int k = 0; k < 3; ++k) { R[k] = t1[k]; R[3 + k] = t2[k]; R[6 + k] = nrm[k]; }
}

// 2-layer laminate (eqs. 5-a, 5-b) by the block formula in the interface frame:
//   A = <C_OO^-1>, B = <C_OO^-1 C_OP>, D = <C_PP - C_PO C_OO^-1 C_OP>
//   C~_OO = A^-1, C~_OP = A^-1 B, C~_PP = D + B^T A^-1 B
// where O are the local components with an index along the normal and P the in-plane ones.
template <typename S>
HOM_HD bool two_layer_t(const S* Ca, const S* Cb, S fa, S fb, const double* nrm, int dim, S* Cout) {
  const int nc = nc_of(dim);
  double R[9], Q[36], QT[36];
  interface_frame(nrm, dim, R);
  mandel_rotation(R, dim, Q);
  for (int i = 0; i < nc; ++i)
    for (int j = 0; j < nc; ++j) QT[i * nc + j] = Q[j * nc + i];
  S tmp[36], La[36], Lb[36];
  matmul_t(Q, Ca, tmp, nc, nc, nc); matmul_t(tmp, QT, La, nc, nc, nc);
  matmul_t(Q, Cb, tmp, nc, nc, nc); matmul_t(tmp, QT, Lb, nc, nc, nc);
  int Pi[3], Oi[3], nP = 0, nO = 0;
  for (int I = 0; I < nc; ++I) {
    int i, j;
    mandel_pair(dim, I, i, j);
    if (i == dim - 1 || j == dim - 1) Oi[nO++] = I; else Pi[nP++] = I;
  }
  S A[9], B[9], D[9];
  for (int a = 0; a < 9; ++a) A[a] = B[a] = D[a] = scal<S>(0.0);
  const S* Ls[2] = {La, Lb};
  const S fs[2] = {fa, fb};
  for (int k = 0; k < 2; ++k) {
    const S* L = Ls[k];
    S OO[9], OP[9], PP[9];
    for (int a = 0; a < nO; ++a)
      for (int b = 0; b < nO; ++b) OO[a * nO + b] = L[Oi[a] * nc + Oi[b]];
    for (int a = 0; a < nO; ++a)
      for (int b = 0; b < nP; ++b) OP[a * nP + b] = L[Oi[a] * nc + Pi[b]];
    for (int a = 0; a < nP; ++a)
      for (int b = 0; b < nP; ++b) PP[a * nP + b] = L[Pi[a] * nc + Pi[b]];
    if (!inv_small_t(OO, nO)) return false;
    S OiOP[9];
    matmul_t(OO, OP, OiOP, nO, nO, nP);
    for (int a = 0; a < nO * nO; ++a) A[a] += fs[k] * OO[a];
    for (int a = 0; a < nO * nP; ++a) B[a] += fs[k] * OiOP[a];
    for (int a = 0; a < nP; ++a)
      for (int b = 0; b < nP; ++b) {
        S s = scal<S>(0.0);
        for (int t = 0; t < nO; ++t) s += OP[t * nP + a] * OiOP[t * nP + b];
        D[a * nP + b] += fs[k] * (PP[a * nP + b] - s);
      }
  }
  if (!inv_small_t(A, nO)) return false;  // A now holds A^-1 = C~_OO
  S AB[9];
  matmul_t(A, B, AB, nO, nO, nP);  // C~_OP
  S loc[36];
  for (int a = 0; a < nO; ++a)
    for (int b = 0; b < nO; ++b) loc[Oi[a] * nc + Oi[b]] = A[a * nO + b];
  for (int a = 0; a < nO; ++a)
    for (int b = 0; b < nP; ++b) {
      loc[Oi[a] * nc + Pi[b]] = AB[a * nP + b];
      loc[Pi[b] * nc + Oi[a]] = AB[a * nP + b];
    }
  for (int a = 0; a < nP; ++a)
    for (int b = 0; b < nP; ++b) {
      S s = scal<S>(0.0);
      for (int t = 0; t < nO; ++t) s += B[t * nP + a] * AB[t * nP + b];
      loc[Pi[a] * nc + Pi[b]] = D[a * nP + b] + s;
    }
  matmul_t(QT, loc, tmp, nc, nc, nc);  // back to the global frame: C = Q^T C' Q
  matmul_t(tmp, Q, Cout, nc, nc, nc);
  return true;
}

// c~ of a mixed ball: rule applied to the phases present (Cs[k], fractions fs[k], k < nph).  A
// 2-layer ball needs nph == 2; without a usable normal it falls back to Voigt.  Returns the rule
// actually applied, or -1 if the 2-layer rule met more than two phases.
template <typename S>
HOM_HD int apply_rule_t(int rule, int nph, const S (*Cs)[36], const S* fs, bool nrm_ok, const double* nrm, int dim,
                        S* Ct) {
  const int nc = nc_of(dim);
  if (rule == HOM_RULE_TWO_LAYER) {
    if (nph != 2) return -1;
    if (!nrm_ok || !two_layer_t(Cs[0], Cs[1], fs[0], fs[1], nrm, dim, Ct)) rule = HOM_RULE_VOIGT;
  }
  if (rule == HOM_RULE_VOIGT) {
    for (int i = 0; i < nc * nc; ++i) {
      S s = scal<S>(0.0);
      for (int k = 0; k < nph; ++k) s += fs[k] * Cs[k][i];
      Ct[i] = s;
    }
  } else if (rule == HOM_RULE_REUSS) {
    S acc[36];
    for (int i = 0; i < nc * nc; ++i) acc[i] = scal<S>(0.0);
    for (int k = 0; k < nph; ++k) {
      S inv[36];
      for (int i = 0; i < nc * nc; ++i) inv[i] = Cs[k][i];
      inv_small_t(inv, nc);
      for (int i = 0; i < nc * nc; ++i) acc[i] += fs[k] * inv[i];
    }
    inv_small_t(acc, nc);
    for (int i = 0; i < nc * nc; ++i) Ct[i] = acc[i];
  }
  return rule;
}

}  // namespace hom

// Eyre-Milton scheme: the per-wave-vector step of its Green pass, shared by the generic passes
// (hom_solver.cu) and the specialised FP32 2D passes (hom_fast2d.cu).
#pragma once

#include "hom_solve_args.cuh"

namespace hom {
namespace {

// the complex operators of hom_common.cuh, also where a translation unit declares others here
using ::hom::operator+;
using ::hom::operator-;
using ::hom::operator*;

__device__ __forceinline__ float em_recip(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double em_recip(double x) { return 1.0 / x; }

// Mandel vector (nc complex entries) <-> symmetric tensor; the shear entries carry sqrt(2).
template <typename T, int DIM, typename V>
__device__ __forceinline__ void mandel_tensor(const V* m, V (&t)[DIM][DIM]) {
  const T rs2 = T(0.707106781186547524400844362105);
  if (DIM == 2) {
    t[0][0] = m[0];
    t[1][1] = m[1];
    t[0][1] = t[1][0] = rs2 * m[2];
  } else {
    t[0][0] = m[0];
    t[1][1] = m[1];
    t[DIM - 1][DIM - 1] = m[2];
    t[1][DIM - 1] = t[DIM - 1][1] = rs2 * m[3];
    t[0][DIM - 1] = t[DIM - 1][0] = rs2 * m[4];
    t[0][1] = t[1][0] = rs2 * m[5];
  }
}
// sym(xi (x) w) in Mandel form
template <typename T, int DIM, typename V>
__device__ __forceinline__ void sym_xi_w(const T* xi, const V* w, V* out) {
  const T rs2 = T(0.707106781186547524400844362105);
  out[0] = xi[0] * w[0];
  out[1] = xi[1] * w[1];
  if (DIM == 2) {
    out[2] = rs2 * (xi[0] * w[1] + xi[1] * w[0]);
  } else {
    out[2] = xi[2] * w[2];
    out[3] = rs2 * (xi[1] * w[2] + xi[2] * w[1]);
    out[4] = rs2 * (xi[0] * w[2] + xi[2] * w[0]);
    out[5] = rs2 * (xi[0] * w[1] + xi[1] * w[0]);
  }
}
// K0(xi)^-1 (s . xi) for a symmetric tensor s: the displacement-like vector whose symmetric
// gradient sym(xi (x) w) is Gamma0(xi) : s (eq. 2)
template <typename T, int DIM, typename V>
__device__ __forceinline__ void kinv_div(const V (&s)[DIM][DIM], const T* xi, T inv_mq, T rq, V* w) {
  V v[DIM];
  V xv = mk(T(0), T(0));
#pragma unroll
  for (int a = 0; a < DIM; ++a) {
    V acc = mk(T(0), T(0));
#pragma unroll
    for (int b = 0; b < DIM; ++b) acc = acc + xi[b] * s[a][b];
    v[a] = acc;
    xv = xv + xi[a] * acc;
  }
#pragma unroll
  for (int a = 0; a < DIM; ++a) w[a] = inv_mq * (v[a] - (rq * xi[a]) * xv);
}

// One wave vector of the Eyre-Milton Green pass.  th: the nc entries of tau_hat (unnormalised DFT),
// uh: the stored u_hat of the current iterate (1/N_v-scaled); un receives the new u_hat (1/N_v-scaled):
// tau_hat - 2 c0 : Gamma0 : tau_hat (k != 0), tau_hat(0) + 2 c0 : E N_v, tau_hat at Nyquist bins.
// With sigma_hat = (N_v u_hat + tau_hat) / 2 and c0 : eps_hat = (N_v u_hat - tau_hat) / 2, accumulates
// (weight 2 for columns whose conjugates are not stored) |sigma_hat . xi|^2, |sigma_hat . xi|^2 /
// |xi|^2 and |eps_hat - Gamma0 : c0 : eps_hat|^2 (k = 0: |eps_hat(0) - N_v E|^2; Nyquist bins:
// |eps_hat|^2).  a0 = lam0 / (2 mu0 + DIM lam0), inv_mu2_0 = 1 / (2 mu0), inv_mu0 = 1 / mu0,
// ratio = (lam0 + mu0) / (lam0 + 2 mu0).
template <typename T, int DIM, typename V>
__device__ __forceinline__ void em_core(const V* th, const V* uh, V* un, const T* xi, bool k0, bool nyq,
                                        bool self_conj, T nvT, T inv_nv, T lam0, T mu2_0, T a0, T inv_mu2_0,
                                        T inv_mu0, T ratio, const double* Eld, Acc<T>& r2acc, Acc<T>& rnacc,
                                        Acc<T>& c2acc) {
  constexpr int NC = DIM == 2 ? 3 : 6;
  V sh[NC], ce[NC], eh[NC];
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    const V nu = nvT * uh[k];
    sh[k] = T(0.5) * (nu + th[k]);  // sigma_hat
    ce[k] = T(0.5) * (nu - th[k]);  // c0 : eps_hat
  }
  {  // eps_hat = c0^-1 : (c0 : eps_hat)
    V tr = mk(T(0), T(0));
#pragma unroll
    for (int k = 0; k < DIM; ++k) tr = tr + ce[k];
#pragma unroll
    for (int k = 0; k < NC; ++k) eh[k] = inv_mu2_0 * (k < DIM ? ce[k] - a0 * tr : ce[k]);
  }
  const T wgt = self_conj ? T(1) : T(2);
  if (k0 || nyq) {
    // k = 0: compatibility residual eps_hat(0) - N_v E, new state tau_hat(0) / N_v + 2 c0 : E.
    // Nyquist bins: Gamma0 is left out: residual eps_hat, new state tau_hat / N_v.
    T c2 = T(0);
    T trE = T(0);
    if (k0)
#pragma unroll
      for (int k = 0; k < DIM; ++k) trE += (T)Eld[k];
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      const V r = k0 ? eh[k] - mk(nvT * (T)Eld[k], T(0)) : eh[k];
      c2 += r.x * r.x + r.y * r.y;
      un[k] = inv_nv * th[k];
      if (k0) un[k].x += T(2) * (mu2_0 * (T)Eld[k] + (k < DIM ? lam0 * trE : T(0)));
    }
    c2acc.add(wgt * c2);
  } else {
    T q2 = T(0);
#pragma unroll
    for (int a = 0; a < DIM; ++a) q2 += xi[a] * xi[a];
    const T inv_q2 = em_recip(q2);
    const T inv_mq = inv_mu0 * inv_q2;
    const T rq = ratio * inv_q2;
    // equilibrium residual of the current iterate: sigma_hat . xi
    V st[DIM][DIM];
    mandel_tensor<T, DIM>(sh, st);
    T r2 = T(0);
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      V r = mk(T(0), T(0));
#pragma unroll
      for (int b = 0; b < DIM; ++b) r = r + xi[b] * st[a][b];
      r2 += r.x * r.x + r.y * r.y;
    }
    r2acc.add(wgt * r2);
    rnacc.add(wgt * r2 * inv_q2);
    // compatibility residual: eps_hat - Gamma0 : (c0 : eps_hat)
    V ct[DIM][DIM], w[DIM], pc[NC];
    mandel_tensor<T, DIM>(ce, ct);
    kinv_div<T, DIM>(ct, xi, inv_mq, rq, w);
    sym_xi_w<T, DIM>(xi, w, pc);
    T c2 = T(0);
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      const V r = eh[k] - pc[k];
      c2 += r.x * r.x + r.y * r.y;
    }
    c2acc.add(wgt * c2);
    // new state: tau_hat - 2 c0 : Gamma0 : tau_hat, scaled by 1/N_v
    V tt[DIM][DIM], gt[NC];
    mandel_tensor<T, DIM>(th, tt);
    kinv_div<T, DIM>(tt, xi, inv_mq, rq, w);
    sym_xi_w<T, DIM>(xi, w, gt);  // Gamma0 : tau_hat
    V tr = mk(T(0), T(0));
#pragma unroll
    for (int k = 0; k < DIM; ++k) tr = tr + gt[k];
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      const V c0g = mu2_0 * gt[k] + (k < DIM ? lam0 * tr : mk(T(0), T(0)));
      un[k] = inv_nv * (th[k] - T(2) * c0g);
    }
  }
}

}  // namespace
}  // namespace hom

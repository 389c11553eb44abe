// Shared device code: complex arithmetic, the in-place mixed-radix FFT used by every pass,
// Mandel helpers and small dense FP64 linear algebra.
//
// FFT scheme.  A length-n line (n = product of radices r_0..r_{m-1}, each 3, 5 or 7) lives in
// shared memory and is transformed in place, one radix stage at a time, with a __syncthreads()
// between stages.  Two orderings are used:
//   * DIT (decimation in time): input at digit-reversed positions P(k), output in natural order;
//     stage s combines r_s sub-transforms of length L_s = r_0...r_{s-1} (twiddle, then DFT_r);
//   * DIF (decimation in frequency): input in natural order, output at positions P(k); stages run
//     in the reverse order (DFT_r, then twiddle).
// Both use the same permutation P, so an inverse DIF followed by a forward DIT needs no reordering
// in between: the row pass does its pointwise constitutive work directly on the permuted data, and
// the Green pass applies Gamma0 to the permuted spectrum.  Butterflies of one stage touch disjoint
// elements, so each thread may process its butterflies one after the other with no extra buffer.
// Twiddles come from a per-length table w[t] = exp(-2 pi i t / n) built on the host in FP64.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hom_dft_consts.h"

#if defined(__CUDA_ARCH__)
#define HOM_LDG(p) __ldg(p)
#else
#define HOM_LDG(p) (*(p))
#endif

#define HOM_HD __host__ __device__ __forceinline__

namespace hom {

constexpr int kMaxStages = 16;
constexpr int kMaxN = 2187;

// ------------------------------------------------------------------ complex arithmetic
template <typename T> struct Cx;
template <> struct Cx<float> { using V = float2; };
template <> struct Cx<double> { using V = double2; };

HOM_HD float2 mk(float x, float y) { return make_float2(x, y); }
HOM_HD double2 mk(double x, double y) { return make_double2(x, y); }
HOM_HD float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
HOM_HD float2 operator-(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
HOM_HD float2 operator*(float s, float2 a) { return make_float2(s * a.x, s * a.y); }
HOM_HD double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
HOM_HD double2 operator-(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
HOM_HD double2 operator*(double s, double2 a) { return make_double2(s * a.x, s * a.y); }

template <typename V> HOM_HD V cmul(V a, V b) { return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
template <typename V> HOM_HD V cmulc(V a, V b) { return mk(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y); }  // a*conj(b)
template <typename V> HOM_HD V conj(V a) { return mk(a.x, -a.y); }
template <typename V> HOM_HD V mul_mi(V a) { return mk(a.y, -a.x); }  // -i * a
template <typename V> HOM_HD V mul_pi(V a) { return mk(-a.y, a.x); }  // +i * a

// ------------------------------------------------------------------ small DFT kernels
// Forward transforms use w = exp(-2 pi i / r); inverse ones use conj(w) (no scaling).
template <bool FWD, typename V, typename T>
HOM_HD void dft3(V* v) {
  const T h = T(0.866025403784438646763723170753);  // sin(2 pi / 3)
  V s = v[1] + v[2];
  V d = v[1] - v[2];
  V m = v[0] - T(0.5) * s;
  v[0] = v[0] + s;
  V t = FWD ? mul_mi(T(h) * d) : mul_pi(T(h) * d);
  v[1] = m + t;
  v[2] = m - t;
}

template <bool FWD, typename V, typename T>
HOM_HD void dft2(V* v) {
  const V s = v[0] + v[1];
  v[1] = v[0] - v[1];
  v[0] = s;
}

template <bool FWD, typename V, typename T>
HOM_HD void dft5(V* v) {
  const T c1 = T(0.309016994374947424102293417183), c2 = T(-0.809016994374947424102293417183);
  const T s1 = T(0.951056516295153572116439333379), s2 = T(0.587785252292473129168705954639);
  V a1 = v[1] + v[4], b1 = v[1] - v[4];
  V a2 = v[2] + v[3], b2 = v[2] - v[3];
  V r1 = v[0] + c1 * a1 + c2 * a2;
  V r2 = v[0] + c2 * a1 + c1 * a2;
  V i1 = s1 * b1 + s2 * b2;
  V i2 = s2 * b1 - s1 * b2;
  v[0] = v[0] + a1 + a2;
  if (FWD) {
    v[1] = r1 + mul_mi(i1); v[4] = r1 + mul_pi(i1);
    v[2] = r2 + mul_mi(i2); v[3] = r2 + mul_pi(i2);
  } else {
    v[1] = r1 + mul_pi(i1); v[4] = r1 + mul_mi(i1);
    v[2] = r2 + mul_pi(i2); v[3] = r2 + mul_mi(i2);
  }
}

template <bool FWD, typename V, typename T>
HOM_HD void dft7(V* v) {
  const T c[4] = {T(1), T(0.623489801858733530525004884004), T(-0.222520933956314404288902564497),
                  T(-0.900968867902419126236102319507)};
  const T s[4] = {T(0), T(0.781831482468029808708444526674), T(0.974927912181823607018131682994),
                  T(0.433883739117558120475768332849)};
  V a[4], b[4];
  for (int q = 1; q <= 3; ++q) { a[q] = v[q] + v[7 - q]; b[q] = v[q] - v[7 - q]; }
  V out[7];
  out[0] = v[0] + a[1] + a[2] + a[3];
  for (int p = 1; p <= 3; ++p) {
    V re = v[0], im = mk(T(0), T(0));
    for (int q = 1; q <= 3; ++q) {
      int k = (p * q) % 7;  // cos/sin of 2 pi k / 7 with the symmetry k -> 7 - k
      T ck = k <= 3 ? c[k] : c[7 - k];
      T sk = k <= 3 ? s[k] : -s[7 - k];
      re = re + ck * a[q];
      im = im + sk * b[q];
    }
    out[p] = FWD ? re + mul_mi(im) : re + mul_pi(im);
    out[7 - p] = FWD ? re + mul_pi(im) : re + mul_mi(im);
  }
  for (int p = 0; p < 7; ++p) v[p] = out[p];
}

// Register DFT of a prime size P >= 11 by symmetric pairs: with a_q = x_q + x_{P-q} and
// b_q = x_q - x_{P-q} (q = 1 .. H, H = (P-1)/2),
//   X_p, X_{P-p} = x_0 + sum_q cos(2 pi pq/P) a_q  -/+  i sum_q sin(2 pi pq/P) b_q   (forward),
// with the signs of the imaginary part swapped for the inverse.  H^2 complex multiply-adds per
// half, against (P-1)^2 for the plain sum.
template <int P, bool FWD, typename V, typename T>
HOM_HD void dft_prime(V* v) {
  constexpr int H = (P - 1) / 2;
  V a[H + 1], b[H + 1];
#pragma unroll
  for (int q = 1; q <= H; ++q) { a[q] = v[q] + v[P - q]; b[q] = v[q] - v[P - q]; }
  V out[P];
  out[0] = v[0];
#pragma unroll
  for (int q = 1; q <= H; ++q) out[0] = out[0] + a[q];
#pragma unroll
  for (int p = 1; p <= H; ++p) {
    V re = v[0], im = mk(T(0), T(0));
#pragma unroll
    for (int q = 1; q <= H; ++q) {
      const int k = (p * q) % P;
      re = re + (T)tw_cos(P, k) * a[q];
      im = im + (T)tw_sin(P, k) * b[q];
    }
    out[p] = FWD ? re + mul_mi(im) : re + mul_pi(im);
    out[P - p] = FWD ? re + mul_pi(im) : re + mul_mi(im);
  }
#pragma unroll
  for (int p = 0; p < P; ++p) v[p] = out[p];
}

// Register DFTs.  dft_small<R> transforms v[0..R) in place; for a composite R the results come
// out in a fixed, compile-time order: X[k] is left in v[out_pos<R>(k)].  Prime radices keep the
// natural order.
template <int R> HOM_HD constexpr int split_a() {  // R = A * B with A the first factor
  return R == 4 ? 2 : R == 8 ? 2 : R == 16 ? 4 : R == 9 ? 3 : R == 15 ? 3 : R == 21 ? 3 : R == 25 ? 5 : R == 27 ? 3 :
         R == 35 ? 5 : R == 45 ? 5 : R == 49 ? 7 : 1;
}
template <int R> HOM_HD constexpr bool is_prime_radix() { return R == 2 || R == 3 || R == 5 || R == 7 || R == 11 || R == 13; }

template <int R> HOM_HD constexpr int out_pos(int k) {
  if constexpr (is_prime_radix<R>()) {
    return k;
  } else {
    constexpr int A = split_a<R>(), B = R / A;
    // block ka = k mod A holds X[ka + A kb] at offset out_pos<B>(kb)
    return B * (k % A) + out_pos<B>(k / A);
  }
}

template <int R, bool FWD, typename V, typename T> HOM_HD void dft_small(V* v);

// Composite register DFT of size R = A * B (Cooley-Tukey inside the registers):
//   X[ka + A kb] = sum_nb w_B^(nb kb) [ w_R^(nb ka) sum_na x[B na + nb] w_A^(na ka) ]
// The inner twiddles w_R^m are compile-time constants once the loops are unrolled.
template <int A, int B, bool FWD, typename V, typename T>
HOM_HD void dft_composite(V* v) {
  constexpr int R = A * B;
#pragma unroll
  for (int nb = 0; nb < B; ++nb) {
    V t[A];
#pragma unroll
    for (int na = 0; na < A; ++na) t[na] = v[B * na + nb];
    dft_small<A, FWD, V, T>(t);
#pragma unroll
    for (int ka = 0; ka < A; ++ka) {
      const V x = t[out_pos<A>(ka)];
      const int m = (nb * ka) % R;
      if (m == 0) {
        v[B * ka + nb] = x;
      } else {
        const V w = mk((T)tw_cos(R, m), FWD ? (T)(-tw_sin(R, m)) : (T)tw_sin(R, m));
        v[B * ka + nb] = cmul(x, w);
      }
    }
  }
#pragma unroll
  for (int ka = 0; ka < A; ++ka) dft_small<B, FWD, V, T>(v + B * ka);
}

template <int R, bool FWD, typename V, typename T>
HOM_HD void dft_small(V* v) {
  if constexpr (R == 2) dft2<FWD, V, T>(v);
  else if constexpr (R == 3) dft3<FWD, V, T>(v);
  else if constexpr (R == 5) dft5<FWD, V, T>(v);
  else if constexpr (R == 7) dft7<FWD, V, T>(v);
  else if constexpr (R == 11 || R == 13) dft_prime<R, FWD, V, T>(v);
  else dft_composite<split_a<R>(), R / split_a<R>(), FWD, V, T>(v);
}

// Exact division by a divisor fixed on the host: q = umulhi(a, m) with m = ceil(2^32 / d) is exact
// whenever a * d < 2^32 (all index ranges here are far below).  Integer division compiled for the
// device goes through int <-> float conversions, which share the slow FP64 pipe on this GPU.
struct FastDiv {
  unsigned m;
  int d;
};
inline FastDiv make_fastdiv(int d) {
  FastDiv f;
  f.d = d;
  f.m = d <= 1 ? 0u : (unsigned)((((unsigned long long)1 << 32) + (unsigned)d - 1) / (unsigned)d);
  return f;
}
HOM_HD int fdiv(int a, const FastDiv& f) {
  if (f.d <= 1) return a;
#if defined(__CUDA_ARCH__)
  return (int)__umulhi((unsigned)a, f.m);
#else
  return (int)(((unsigned long long)(unsigned)a * f.m) >> 32);
#endif
}

// Enumerates the flat indices f = tid, tid + step, ... < total as pairs (a, b) with f = a * nb + b,
// updating the pair with carries instead of dividing.
struct Iter2 {
  int a, b, da, db, nb;
  HOM_HD Iter2(int f0, int step, const FastDiv& div) : nb(div.d) {
    a = fdiv(f0, div);
    b = f0 - a * nb;
    da = fdiv(step, div);
    db = step - da * nb;
  }
  HOM_HD void next() {
    b += db;
    a += da;
    if (b >= nb) { b -= nb; ++a; }
  }
};

// ------------------------------------------------------------------ FFT plan
// Device-resident description of the transform of one length.
struct Plan {
  int n;
  int nstage;
  int radix[kMaxStages];  // DIT order
  int span[kMaxStages];   // L_s = radix[0] * ... * radix[s-1]
  FastDiv div_nb[kMaxStages];  // n / radix[s] (butterflies per line)
  FastDiv div_L[kMaxStages];   // span[s]
  FastDiv div_n, div_h;        // n and n / 2 + 1 (the half spectrum of a real line)
  const uint16_t* perm;   // perm[k] = position of index k in the digit-reversed layout
  const float2* tw32;     // exp(-2 pi i t / n), t < n
  const double2* tw64;
  const float* xi32;      // 2 pi a(k): signed DFT frequency of bin k times 2 pi
  const double* xi64;
  const float2* rot32;    // (2n sin(pi a/n), cos(pi a/n)): the rotated scheme's wave-vector factors
  const double2* rot64;
};

// Fills the dividers of a plan whose n, nstage, radix and span are set.
inline void plan_dividers(Plan& p) {
  for (int s = 0; s < p.nstage; ++s) {
    p.div_nb[s] = make_fastdiv(p.n / p.radix[s]);
    p.div_L[s] = make_fastdiv(p.span[s]);
  }
  p.div_n = make_fastdiv(p.n);
  p.div_h = make_fastdiv(p.n / 2 + 1);
}

template <typename V> HOM_HD const V* twiddles(const Plan& p);
template <> HOM_HD const float2* twiddles<float2>(const Plan& p) { return p.tw32; }
template <> HOM_HD const double2* twiddles<double2>(const Plan& p) { return p.tw64; }

// One DIT stage (radix R, span L) over `nl` lines of length n stored back to back (line stride
// `ls` elements).  Thread `tid` of `nthr` handles butterflies tid, tid + nthr, ... (a butterfly is
// (line, block, j) with j < L), enumerated with carries.  `tw` is the length-n twiddle table.
template <int R, bool FWD, typename V, typename T>
HOM_HD void dit_stage(V* s, int nl, int ls, int n, int L, const V* tw, int tid, int nthr, const FastDiv& dnb,
                      const FastDiv& dL) {
  const int B = L * R;
  const int nb = n / R;           // butterflies per line
  const int nblk = fdiv(nb, dL);  // n / B blocks per line, also the twiddle stride
  const int twstep = nblk;
  Iter2 lw(tid, nthr, dnb);       // (line, w)
  Iter2 bj(lw.b, lw.db, dL);      // (block, j) of w; advanced by the same step
  for (; lw.a < nl; ) {
    V* base = s + lw.a * ls + bj.a * B + bj.b;
    const int j = bj.b;
    V v[R];
    v[0] = base[0];
#pragma unroll
    for (int q = 1; q < R; ++q) {
      V x = base[q * L];
      if (L > 1) {
        V t = tw[j * q * twstep];
        x = FWD ? cmul(x, t) : cmulc(x, t);
      }
      v[q] = x;
    }
    dft_small<R, FWD, V, T>(v);
#pragma unroll
    for (int p = 0; p < R; ++p) base[p * L] = v[out_pos<R>(p)];
    // advance (line, w) and (block, j) together
    lw.b += lw.db;
    lw.a += lw.da;
    bj.next();
    if (bj.a >= nblk) bj.a -= nblk;
    if (lw.b >= nb) {
      lw.b -= nb;
      ++lw.a;
    }
  }
}

// One DIF stage (radix R, span L): DFT_r of the inputs, then the twiddles, written in place.
template <int R, bool FWD, typename V, typename T>
HOM_HD void dif_stage(V* s, int nl, int ls, int n, int L, const V* tw, int tid, int nthr, const FastDiv& dnb,
                      const FastDiv& dL) {
  const int B = L * R;
  const int nb = n / R;
  const int nblk = fdiv(nb, dL);
  const int twstep = nblk;
  Iter2 lw(tid, nthr, dnb);
  Iter2 bj(lw.b, lw.db, dL);
  for (; lw.a < nl; ) {
    V* base = s + lw.a * ls + bj.a * B + bj.b;
    const int j = bj.b;
    V v[R];
#pragma unroll
    for (int q = 0; q < R; ++q) v[q] = base[q * L];
    dft_small<R, FWD, V, T>(v);
    base[0] = v[0];
#pragma unroll
    for (int p = 1; p < R; ++p) {
      V x = v[out_pos<R>(p)];
      if (L > 1) {
        V t = tw[j * p * twstep];
        x = FWD ? cmul(x, t) : cmulc(x, t);
      }
      base[p * L] = x;
    }
    lw.b += lw.db;
    lw.a += lw.da;
    bj.next();
    if (bj.a >= nblk) bj.a -= nblk;
    if (lw.b >= nb) {
      lw.b -= nb;
      ++lw.a;
    }
  }
}

#if defined(__CUDA_ARCH__)
#define HOM_SYNC() __syncthreads()
#else
#define HOM_SYNC() ((void)0)
#endif

// Radix dispatch of one stage; MAXR bounds the register radices compiled into a kernel (the
// register footprint of a kernel is set by its largest radix).
#define HOM_RADIX_CASES(STAGE)                                              \
  switch (r) {                                                              \
    case 2: STAGE(2); break;                                                \
    case 3: STAGE(3); break;                                                \
    case 4: STAGE(4); break;                                                \
    case 5: STAGE(5); break;                                                \
    case 7: STAGE(7); break;                                                \
    case 8: STAGE(8); break;                                                \
    case 9: if constexpr (MAXR >= 9) STAGE(9); break;                       \
    case 11: if constexpr (MAXR >= 11) STAGE(11); break;                    \
    case 13: if constexpr (MAXR >= 13) STAGE(13); break;                    \
    case 15: if constexpr (MAXR >= 15) STAGE(15); break;                    \
    case 16: if constexpr (MAXR >= 16) STAGE(16); break;                    \
    case 21: if constexpr (MAXR >= 21) STAGE(21); break;                    \
    case 25: if constexpr (MAXR >= 25) STAGE(25); break;                    \
    case 27: if constexpr (MAXR >= 27) STAGE(27); break;                    \
    case 35: if constexpr (MAXR >= 35) STAGE(35); break;                    \
    case 45: if constexpr (MAXR >= 45) STAGE(45); break;                    \
    case 49: if constexpr (MAXR >= 49) STAGE(49); break;                    \
    default: break;                                                         \
  }

// Whole transforms.  Must be called by every thread of the block (they contain barriers).
// `tw` is the length-n twiddle table (shared memory in the kernels).  The plan's radices must
// not exceed MAXR.
template <bool FWD, int MAXR, typename V, typename T>
HOM_HD void fft_dit(V* s, int nl, int ls, const Plan& p, const V* tw, int tid, int nthr) {
  for (int st = 0; st < p.nstage; ++st) {
    const int r = p.radix[st], L = p.span[st];
#define HOM_DIT(R) dit_stage<R, FWD, V, T>(s, nl, ls, p.n, L, tw, tid, nthr, p.div_nb[st], p.div_L[st])
    HOM_RADIX_CASES(HOM_DIT)
#undef HOM_DIT
    HOM_SYNC();
  }
}

template <bool FWD, int MAXR, typename V, typename T>
HOM_HD void fft_dif(V* s, int nl, int ls, const Plan& p, const V* tw, int tid, int nthr) {
  for (int st = p.nstage - 1; st >= 0; --st) {
    const int r = p.radix[st], L = p.span[st];
#define HOM_DIF(R) dif_stage<R, FWD, V, T>(s, nl, ls, p.n, L, tw, tid, nthr, p.div_nb[st], p.div_L[st])
    HOM_RADIX_CASES(HOM_DIF)
#undef HOM_DIF
    HOM_SYNC();
  }
}

// ------------------------------------------------------------------ Mandel helpers
HOM_HD int nc_of(int dim) { return dim == 2 ? 3 : 6; }
HOM_HD int ns_of(int dim) { return dim == 2 ? 6 : 21; }
// Index pairs (i, j) of Mandel component I.
HOM_HD void mandel_pair(int dim, int I, int& i, int& j) {
  if (dim == 2) {
    const int a[3] = {0, 1, 0}, b[3] = {0, 1, 1};
    i = a[I]; j = b[I];
  } else {
    const int a[6] = {0, 1, 2, 1, 0, 0}, b[6] = {0, 1, 2, 2, 2, 1};
    i = a[I]; j = b[I];
  }
}
// Position of (I, J) in the packed upper triangle of an nc x nc matrix.
HOM_HD int packed_index(int nc, int I, int J) {
  if (I > J) { int t = I; I = J; J = t; }
  return I * nc - I * (I - 1) / 2 + (J - I);
}

}  // namespace hom

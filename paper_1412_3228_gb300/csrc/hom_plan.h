// Host-side construction of FFT plans: radix factorisation, digit-reversal permutation and
// the FP64 twiddle table w[t] = exp(-2 pi i t / n) (rounded to FP32 for the FP32 path).
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <functional>
#include <utility>
#include <vector>

namespace hom {

struct HostPlan {
  int n = 0;
  std::vector<int> radix;       // DIT order
  std::vector<int> span;        // product of the radices before each stage
  std::vector<uint16_t> perm;   // position of index k in the digit-reversed layout
  std::vector<double> tw;       // interleaved (re, im) of exp(-2 pi i t / n)
  std::vector<double> xi;       // 2 pi a(k), a(k) the signed frequency of DFT bin k
  std::vector<double> rot;      // interleaved (2n sin(pi a/n), cos(pi a/n)): factors of the rotated
                                // scheme's wave vector q_j = 2n sin(pi a_j/n) prod_{m!=j} cos(pi a_m/n)
};

// Factor n into the register radices {2, 3, 4, 5, 7, 8, 9, 11, 13, 15, 16, 21, 25, 27, 35, 45, 49}
// (each at most `max_radix`) with the fewest stages, then the smallest largest radix.  Returns
// false if n has a prime factor other than 2, 3, 5, 7, 11, 13.
inline bool factorize(int n, std::vector<int>& radix, int max_radix = 45) {
  static const int kRadices[] = {45, 35, 27, 25, 21, 16, 15, 13, 11, 9, 8, 7, 5, 4, 3, 2, 49};
  radix.clear();
  if (n < 3) return false;
  int m = n;
  for (int r : {2, 3, 5, 7, 11, 13})
    while (m % r == 0) m /= r;
  if (m != 1) return false;
  std::vector<int> best, cur;
  std::function<void(int)> search = [&](int rem) {
    if (rem == 1) {
      auto key = [](const std::vector<int>& v) {
        int mx = 0;
        for (int r : v) mx = std::max(mx, r);
        return std::make_pair((int)v.size(), mx);
      };
      if (best.empty() || key(cur) < key(best)) best = cur;
      return;
    }
    if (!best.empty() && (int)cur.size() + 1 > (int)best.size()) return;
    for (int r : kRadices) {
      if (r > max_radix || rem % r != 0) continue;
      if (!cur.empty() && r > cur.back()) continue;  // non-increasing order: one ordering per multiset
      cur.push_back(r);
      search(rem / r);
      cur.pop_back();
    }
  };
  search(n);
  radix = best;
  return !radix.empty();
}

// Plan tables for a given radix list (DIT order); the product of the radices must be n.
inline bool build_host_plan_radices(int n, const std::vector<int>& radix, HostPlan& p) {
  p.n = n;
  p.radix = radix;
  int prod = 1;
  for (int r : radix) prod *= r;
  if (prod != n || radix.empty()) return false;
  const int m = (int)p.radix.size();
  p.span.assign(m, 1);
  for (int s = 1; s < m; ++s) p.span[s] = p.span[s - 1] * p.radix[s - 1];
  // P(k): the last DIT stage splits k = d + r k' into block d of length n/r, recursively.
  p.perm.assign(n, 0);
  for (int k = 0; k < n; ++k) {
    int pos = 0, kk = k, len = n;
    for (int s = m - 1; s >= 0; --s) {
      const int r = p.radix[s];
      len /= r;
      pos += (kk % r) * len;
      kk /= r;
    }
    p.perm[k] = (uint16_t)pos;
  }
  p.xi.assign(n, 0.0);
  // signed frequency of bin k: k up to n / 2 (the Nyquist bin of an even grid counts as +n/2), else k - n
  for (int k = 0; k < n; ++k) p.xi[k] = 6.28318530717958647692528676656 * (double)(k <= n / 2 ? k : k - n);
  p.rot.assign(2 * (size_t)n, 0.0);
  for (int k = 0; k < n; ++k) {
    const double h = 3.14159265358979323846264338328 * (double)(k <= n / 2 ? k : k - n) / (double)n;
    p.rot[2 * k] = 2.0 * n * std::sin(h);
    p.rot[2 * k + 1] = std::cos(h);
  }
  p.tw.assign(2 * (size_t)n, 0.0);
  const double two_pi = 6.28318530717958647692528676656;
  for (int t = 0; t < n; ++t) {
    // angle reduced to [0, 2 pi) exactly in integers before the FP64 evaluation
    const double a = two_pi * (double)t / (double)n;
    p.tw[2 * t] = std::cos(a);
    p.tw[2 * t + 1] = -std::sin(a);
  }
  return true;
}

inline bool build_host_plan(int n, HostPlan& p, int max_radix = 45) {
  std::vector<int> radix;
  if (!factorize(n, radix, max_radix)) return false;
  return build_host_plan_radices(n, radix, p);
}

// Device layout of a plan's tables (each block 256-byte aligned): permutation (uint16),
// FP32 twiddles, FP64 twiddles, FP32 wave numbers, FP64 wave numbers, FP32 and FP64 factors of the
// rotated scheme's wave vector.
inline size_t plan_table_bytes(int n) {
  auto up = [](size_t b) { return (b + 255) / 256 * 256; };
  return up((size_t)n * 2) + up((size_t)n * 8) + up((size_t)n * 16) + up((size_t)n * 4) + up((size_t)n * 8) +
         up((size_t)n * 8) + up((size_t)n * 16);
}

inline void fill_plan_tables(const HostPlan& hp, unsigned char* dst) {
  auto up = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t n = (size_t)hp.n;
  unsigned char* q = dst;
  std::memcpy(q, hp.perm.data(), n * sizeof(uint16_t));
  q += up(n * 2);
  float* t32 = reinterpret_cast<float*>(q);
  for (size_t t = 0; t < n; ++t) { t32[2 * t] = (float)hp.tw[2 * t]; t32[2 * t + 1] = (float)hp.tw[2 * t + 1]; }
  q += up(n * 8);
  std::memcpy(q, hp.tw.data(), n * 16);
  q += up(n * 16);
  float* x32 = reinterpret_cast<float*>(q);
  for (size_t k = 0; k < n; ++k) x32[k] = (float)hp.xi[k];
  q += up(n * 4);
  std::memcpy(q, hp.xi.data(), n * 8);
  q += up(n * 8);
  float* r32 = reinterpret_cast<float*>(q);
  for (size_t k = 0; k < 2 * n; ++k) r32[k] = (float)hp.rot[k];
  q += up(n * 8);
  std::memcpy(q, hp.rot.data(), n * 16);
}

}  // namespace hom

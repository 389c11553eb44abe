// Host-side check of the generic mixed-radix FFT (the templates of hom_common.cuh compile for the
// host too): for every supported length n in [lo, hi] (odd and even), the DIF transform of natural-order input
// and the DIT transform of digit-reversed input are compared with a long-double DFT at sampled bins,
// under several thread schedules.  A schedule runs the threads of one stage one after another and
// separates stages, which is what the kernels' barriers guarantee; butterflies of one stage touch
// disjoint elements, so any interleaving inside a stage gives the same result.
//
//   fft_host_check lo hi [max_radix]   -> prints failing lengths, "ok" or "FAIL" at the end, exit 0/1
// max_radix (default 45) bounds the register radices of the plans, as the kernels' MAXR does
// (FP64 kernels use plans up to radix 15, FP32 ones up to 27 or 45).
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <random>
#include <vector>

#include "../paper_1412_3228_gb300/csrc/hom_internal.h"
#include "../paper_1412_3228_gb300/csrc/hom_plan.h"

using namespace hom;

template <bool FWD>
static void run_dif(std::vector<double2>& a, const Plan& p, const std::vector<double2>& tw, int nthr) {
  for (int st = p.nstage - 1; st >= 0; --st) {
    const int r = p.radix[st], L = p.span[st];
    for (int tid = 0; tid < nthr; ++tid) {
      constexpr int MAXR = 49;
#define HOM_DIF(R) dif_stage<R, FWD, double2, double>(a.data(), 1, p.n, p.n, L, tw.data(), tid, nthr, p.div_nb[st], p.div_L[st])
      HOM_RADIX_CASES(HOM_DIF)
#undef HOM_DIF
    }
  }
}

template <bool FWD>
static void run_dit(std::vector<double2>& a, const Plan& p, const std::vector<double2>& tw, int nthr) {
  for (int st = 0; st < p.nstage; ++st) {
    const int r = p.radix[st], L = p.span[st];
    for (int tid = 0; tid < nthr; ++tid) {
      constexpr int MAXR = 49;
#define HOM_DIT(R) dit_stage<R, FWD, double2, double>(a.data(), 1, p.n, p.n, L, tw.data(), tid, nthr, p.div_nb[st], p.div_L[st])
      HOM_RADIX_CASES(HOM_DIT)
#undef HOM_DIT
    }
  }
}

int main(int argc, char** argv) {
  const int lo = argc > 1 ? atoi(argv[1]) : 3, hi = argc > 2 ? atoi(argv[2]) : 2187;
  const int max_radix = argc > 3 ? atoi(argv[3]) : 45;
  std::mt19937 gen(12345);
  std::uniform_real_distribution<double> u(-1.0, 1.0);
  int bad = 0, checked = 0;
  for (int n = lo; n <= hi; ++n) {
    std::vector<int> radices;
    if (!factorize(n, radices) || (int)radices.size() > kMaxStages) continue;
    HostPlan hp;
    if (!build_host_plan(n, hp, max_radix)) { printf("n %d: no plan up to radix %d\n", n, max_radix); ++bad; continue; }
    Plan p{};
    p.n = n;
    p.nstage = (int)hp.radix.size();
    for (int s = 0; s < p.nstage; ++s) { p.radix[s] = hp.radix[s]; p.span[s] = hp.span[s]; }
    plan_dividers(p);
    std::vector<double2> tw(n), x(n);
    for (int t = 0; t < n; ++t) tw[t] = make_double2(hp.tw[2 * t], hp.tw[2 * t + 1]);
    for (auto& v : x) v = make_double2(u(gen), u(gen));
    // sampled bins: the first and last few, and a stride through the middle
    std::vector<int> bins;
    for (int k = 0; k < n; k += (n > 64 ? n / 29 : 1)) bins.push_back(k);
    bins.push_back(n - 1);
    double worst = 0.0;
    for (int fwd = 0; fwd < 2; ++fwd) {
      std::vector<long double> re(n), im(n);
      for (int k : bins) {
        long double sr = 0, si = 0;
        for (int j = 0; j < n; ++j) {
          const long double ang = (fwd ? -2.0L : 2.0L) * 3.14159265358979323846264338327950288L *
                                  (long double)((long long)j * k % n) / (long double)n;
          sr += x[j].x * cosl(ang) - x[j].y * sinl(ang);
          si += x[j].x * sinl(ang) + x[j].y * cosl(ang);
        }
        re[k] = sr;
        im[k] = si;
      }
      for (int nthr : {1, 7, 256}) {
        std::vector<double2> a = x, b(n);
        for (int k = 0; k < n; ++k) b[hp.perm[k]] = x[k];
        if (fwd) { run_dif<true>(a, p, tw, nthr); run_dit<true>(b, p, tw, nthr); }
        else { run_dif<false>(a, p, tw, nthr); run_dit<false>(b, p, tw, nthr); }
        for (int k : bins) {
          const double2 d = a[hp.perm[k]], e = b[k];
          worst = fmax(worst, fmax(fabs(d.x - (double)re[k]), fabs(d.y - (double)im[k])));
          worst = fmax(worst, fmax(fabs(e.x - (double)re[k]), fabs(e.y - (double)im[k])));
        }
      }
    }
    // FP64 butterflies: error grows like sqrt(n) log n times the unit roundoff on O(sqrt(n)) values
    const double tol = 1e-13 * std::sqrt((double)n) * std::log((double)n + 1.0) + 1e-14;
    ++checked;
    if (!(worst <= tol)) {
      ++bad;
      printf("n %d radices", n);
      for (int r : hp.radix) printf(" %d", r);
      printf(": max error %.3e > %.3e\n", worst, tol);
    }
  }
  printf("%d lengths checked, %d failed\n%s\n", checked, bad, bad ? "FAIL" : "ok");
  return bad ? 1 : 0;
}

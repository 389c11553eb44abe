// Conjugate gradients on the passes of the basic scheme.  An accelerated scheme of the kind the
// paper's introduction and section 5 call complementary to filtering (its refs. [3, 12]), applied
// to the same discrete problem: find eps = E + x, x compatible with zero mean, such that
// G(c~ : eps) = 0, where G is the L2-orthogonal projection onto compatible zero-mean fields
// (eq. (2)'s Green operator for an isotropic reference medium c0 = s I, times s).
//
// With c0 = s I (lambda0 = 0, mu0 = s/2) and zero mean strain, one row pass + Green pass applied to
// a compatible zero-mean field p returns
//     p' = -Gamma0 * ((c~ - s I) : p) = p - G(c~ : p) / s,
// so the CG operator A p = G(c~ : p) is q = s (p - p') and costs no new transform.  s is the
// smallest eigenvalue of the cell's phase stiffnesses (a lower bound for every filtered c~ too):
// then |p - p'| >= |p|, and the subtraction loses no digits even where c~ is tiny (a compliant
// inclusion).  Applied to the uniform field E the passes return b / s with b = -G(c~ : E), the
// first residual; applied to E + x they return x - G(c~ : (E + x)) / s, whence the true residual.
// The row pass's per-task sums of sigma give <c~ : p>, so the mean stress is tracked by linearity
// (and recomputed exactly at each verification).  Per (cell, load) pair:
//     start:  r = b, x = 0, p = r (p lives in the eps buffer the next row pass reads)
//     step:   q = A p;  alpha = <r,r>/<p,q>;  x += alpha p;  r -= alpha q;  <sigma> += alpha <c~:p>
//             beta = <r,r>_new/<r,r>;  p = r + beta p
//     stop:   e_G = sqrt(<r,r>/N_v) / |<sigma>| < tol, then one verification pass on E + x: the
//             pair stops if the true residual passes too, else CG restarts from it (p = r)
// e_n <= e_G <= sqrt2 e_n.  The verification state of a pair (vmode): 0 CG step, 1 the pass runs on
// E + x, 2 restart after a failed verification.
//
// The fields stay in the solver's mixed domain (x-spectrum of each real row, generic layout
// [cell][load][z][y][kx][component]).  The stored spectrum is (1/n) x DFT, so by Parseval the real
// inner product of two fields is n sum_rows sum_comp (U_0 V_0 + 2 sum_{0<kx<H} Re U_kx conj V_kx);
// the factor n is applied where absolute sizes matter (the stopping rule).
#pragma once

#include "hom_solve_args.cuh"

namespace hom {

struct CgArgs {
  void* x;         // [ws elements] compatible part of the strain
  void* r;         // [ws elements] residual
  double* part;    // [npairs][nchunk] per-CTA partial inner products
  double* rr;      // [npairs] <r, r> (spectral weighting, without the factor n)
  double* alpha;   // [npairs]
  double* beta;    // [npairs]
  double* ssum;    // [npairs][nc] sum over voxels of the iterate's stress
  int* vmode;      // [npairs] verification state (0 step, 1 verify, 2 restart)
  int* steps;      // [npairs] CG steps taken
  const double* E; // [npairs][nc] macroscopic strains (the passes themselves run with zero mean strain)
  int nchunk;      // CTAs per pair in the element kernels (grid.y)
};

constexpr int kCgThreads = 256;
constexpr int kCgElems = 8192;  // complex elements per CTA (rounded to whole rows)

// Rows per CTA of the element kernels for a cell whose rows hold Hp * nc complex elements.
__host__ __device__ inline int cg_rows_per_cta(int Hp, int nc) {
  const int r = kCgElems / (Hp * nc);
  return r > 0 ? r : 1;
}

enum CgStage { kCgStart = 0, kCgPq = 1, kCgUpdate = 2, kCgDir = 3, kCgFinal = 4 };

// Element kernels over one pair's mixed-domain fields, grid (npairs, nchunk).
//   kCgStart:  r = p = s p' (the start pass on E left b / s in eps[1]; p overwrites it); x = 0;
//              sum <r, r>
//   kCgPq:     vmode 0: sum <p, q> with q = s (p - p');  vmode 1: r = s (p' - x), sum <r, r>
//   kCgUpdate: vmode 0: x += alpha p;  r -= alpha q;  sum <r, r>
//   kCgDir:    vmode 0 or 2: p = r + beta p;  vmode 1: E + x (the verification input)
//              (runs after the control advanced the iteration counter)
//   kCgFinal:  eps[iters & 1] = E + x for the output pass (every pair)
// Divider by d for Iter2 (computed once per CTA: one 64-bit division).
__device__ __forceinline__ FastDiv make_fastdiv_dev(int d) {
  FastDiv f;
  f.d = d;
  f.m = d <= 1 ? 0u : (unsigned)((((unsigned long long)1 << 32) + (unsigned)d - 1) / (unsigned)d);
  return f;
}

// Running sum of the element kernels: Kahan-compensated in FP32; plain in FP64 (at most a few
// dozen terms per thread, and FP64 arithmetic is scarce on this GPU).
template <typename T> struct CgSum {
  Acc<T> a;
  __device__ __forceinline__ void add(T x) { a.add(x); }
};
template <> struct CgSum<double> {
  Acc<double> a;
  __device__ __forceinline__ void add(double x) { a.s += x; }
};

template <typename T, int DIM, int STAGE>
__global__ void __launch_bounds__(kCgThreads) k_cg_elems(SolveArgs A, CgArgs G) {
  using V = typename Cx<T>::V;
  constexpr int NC = DIM == 2 ? 3 : 6;
  const int pair = blockIdx.x;
  if (STAGE != kCgFinal && !A.active[pair]) return;
  const int vm = STAGE == kCgFinal ? 0 : G.vmode[pair];
  if (STAGE == kCgUpdate && vm != 0) return;
  const PairDev pr = A.pairs[pair];
  const CellDev c = A.cells[pr.cell];
  const int rowlen = c.Hp * NC;
  const int rpc = cg_rows_per_cta(c.Hp, NC);
  const int row0 = blockIdx.y * rpc;
  const int it = *A.it_dev;
  double* part = G.part + (size_t)pair * G.nchunk + blockIdx.y;
  if (row0 >= c.nrows) {
    if (STAGE != kCgDir && STAGE != kCgFinal && threadIdx.x == 0) *part = 0.0;
    return;
  }
  const int nrow = min(rpc, c.nrows - row0);
  const size_t base = c.ws_off + ((size_t)pr.load * c.nrows + row0) * rowlen;
  // kCgDir runs after the counter advanced: the old p is in eps[(it + 1) & 1], the output goes to
  // eps[it & 1]; every other stage reads p from eps[it & 1] and the pass output p' from eps[(it + 1) & 1]
  const V* pv = static_cast<const V*>(A.eps[STAGE == kCgDir ? ((it + 1) & 1) : (it & 1)]) + base;
  const V* fv = static_cast<const V*>(A.eps[(it + 1) & 1]) + base;
  V* xv = static_cast<V*>(G.x) + base;
  V* rv = static_cast<V*>(G.r) + base;
  const T sc = (T)(2.0 * c.mu0);  // s of the reference medium c0 = s I
  // the update folds s into the step: r -= (alpha s) (p - p')
  const T a = STAGE == kCgUpdate ? (T)G.alpha[pair] : T(0);
  const T as = STAGE == kCgUpdate ? (T)(G.alpha[pair] * 2.0 * c.mu0) : T(0);
  const T b = STAGE == kCgDir ? (T)G.beta[pair] : T(0);
  V* outp = static_cast<V*>(A.eps[STAGE == kCgFinal ? (A.iters[pair] & 1) : STAGE == kCgStart ? ((it + 1) & 1) : (it & 1)]) +
            base;
  const double* Eld = G.E + (size_t)pair * NC;
  const bool write_state = STAGE == kCgFinal || (STAGE == kCgDir && vm == 1);
  const V zero = mk(T(0), T(0));
  // Sums over the row positions: kx = 0 entries count once, 0 < kx < H twice (Parseval for the
  // half spectrum), padding kx >= H not at all; kept as sum_all and sum_kx0 (total = 2 all - kx0).
  CgSum<T> acc_all, acc_0;
  // (row, position) pairs enumerated with carries (no division per element)
  const FastDiv drow = make_fastdiv_dev(rowlen);
  for (Iter2 e(threadIdx.x, kCgThreads, drow); e.a < nrow; e.next()) {
    const int j = e.b;                           // position in the row: kx * NC + component
    const size_t f = (size_t)e.a * rowlen + j;
    if (j >= c.H * NC) {  // row padding: never read by the passes; kept at zero in the CG fields
      if (STAGE == kCgStart) { rv[f] = zero; xv[f] = zero; outp[f] = zero; }
      else if (STAGE == kCgDir || STAGE == kCgFinal) outp[f] = zero;
      continue;
    }
    T term = T(0);
    if (STAGE == kCgStart) {
      const V pp = fv[f];
      const V r = mk(sc * pp.x, sc * pp.y);
      rv[f] = r;
      outp[f] = r;  // p = r, in the buffer the next row pass reads
      xv[f] = zero;
      term = r.x * r.x + r.y * r.y;
    } else if (STAGE == kCgPq) {
      const V pp = fv[f];
      if (vm == 1) {  // true residual of E + x
        const V x = xv[f];
        const V r = mk(sc * (pp.x - x.x), sc * (pp.y - x.y));
        rv[f] = r;
        term = r.x * r.x + r.y * r.y;
      } else {  // <p, p - p'> (times s in the control)
        const V p = pv[f];
        term = p.x * (p.x - pp.x) + p.y * (p.y - pp.y);
      }
    } else if (STAGE == kCgUpdate) {
      const V p = pv[f], pp = fv[f];
      V x = xv[f], r = rv[f];
      x = mk(x.x + a * p.x, x.y + a * p.y);
      r = mk(r.x - as * (p.x - pp.x), r.y - as * (p.y - pp.y));
      xv[f] = x;
      rv[f] = r;
      term = r.x * r.x + r.y * r.y;
    } else if (!write_state) {  // kCgDir, vmode 0 or 2
      const V p = pv[f], r = rv[f];
      outp[f] = mk(r.x + b * p.x, r.y + b * p.y);
    } else {  // E + x
      V x = xv[f];
      if (j < NC) x.x += (T)Eld[j];
      outp[f] = x;
    }
    if (STAGE != kCgDir && STAGE != kCgFinal) {
      acc_all.add(term);
      if (j < NC) acc_0.add(term);
    }
  }
  if (STAGE == kCgDir || STAGE == kCgFinal) return;
  const Acc<T> vv[2] = {acc_all.a, acc_0.a};
  double tot[2];
  block_sum<T, 2, kCgThreads>(vv, tot);
  if (threadIdx.x == 0) *part = (2.0 * tot[0] - tot[1]) * (STAGE == kCgPq && vm != 1 ? (double)sc : 1.0);
}

// Per-pair control, one CTA per pair (fixed-order FP64 sums: deterministic).
//   kCgStart:  <r,r> and the mean stress of E from the start pass; stopping test at 0 steps
//   kCgPq:     alpha = <r,r>/<p,q>; <sigma> += alpha <c~ : p>
//   kCgUpdate: beta, stopping test after the step
// The stopping stages count the active pairs and advance the iteration counter (last CTA).
constexpr int kCgCtlThreads = 128;
template <int STAGE>
__global__ void __launch_bounds__(kCgCtlThreads) k_cg_control(SolveArgs A, CgArgs G, int nc) {
  __shared__ bool s_last;
  __shared__ double s_red[kCgCtlThreads / 32][7];
  __shared__ int s_cnt[kCgCtlThreads / 32];
  const int pair = blockIdx.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int it = *A.it_dev;
  if (A.active[pair]) {
    const PairDev pr = A.pairs[pair];
    const CellDev c = A.cells[pr.cell];
    const int nchunk = (c.nrows + cg_rows_per_cta(c.Hp, nc) - 1) / cg_rows_per_cta(c.Hp, nc);
    // v[0]: inner product, v[1..nc]: stress sums of the last row pass
    double v[7];
#pragma unroll
    for (int k = 0; k < 7; ++k) v[k] = 0.0;
    for (int b = threadIdx.x; b < nchunk; b += kCgCtlThreads) v[0] += G.part[(size_t)pair * G.nchunk + b];
    if (STAGE != kCgUpdate)
      for (int tk = pr.rtask0 + (int)threadIdx.x; tk < pr.rtask1; tk += kCgCtlThreads) {
        const double* p = A.partR + ((size_t)tk * A.L + pr.load) * nc;
        for (int k = 0; k < nc; ++k) v[1 + k] += p[k];
      }
#pragma unroll
    for (int k = 0; k < 7; ++k)
      for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    if (lane == 0)
#pragma unroll
      for (int k = 0; k < 7; ++k) s_red[wid][k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0) {
      double sum[7];
      for (int k = 0; k < 7; ++k) {
        sum[k] = 0.0;
        for (int w = 0; w < kCgCtlThreads / 32; ++w) sum[k] += s_red[w][k];
      }
      double* ss = G.ssum + (size_t)pair * nc;
      const int vm = G.vmode[pair];
      // e_G of the pair's residual sum rr (spectral weighting) and stress sum: sqrt(n rr / N_v) / |<sigma>|
      auto e_of = [&](double rr) {
        double s2 = 0.0;
        for (int k = 0; k < nc; ++k) s2 += ss[k] * ss[k];
        return sqrt((double)c.n * rr / (double)c.nv) * (double)c.nv / sqrt(s2);
      };
      auto publish = [&](double eg) {
        for (int k = 0; k < nc; ++k) A.mean_sigma[(size_t)pair * nc + k] = ss[k] / (double)c.nv;
        A.err[pair] = eg;
        A.errn[pair] = eg;
      };
      int st = -1;
      if (STAGE == kCgStart) {
        // the first residual is exact: no verification needed
        G.rr[pair] = sum[0];
        for (int k = 0; k < nc; ++k) ss[k] = sum[1 + k];
        G.steps[pair] = 0;
        const double eg = e_of(sum[0]);
        publish(eg);
        if (!isfinite(eg)) st = HOM_STATUS_DIVERGED;
        else if (eg < A.tol) st = HOM_STATUS_CONVERGED;
        else if (A.max_iter <= 0) st = HOM_STATUS_MAX_ITER;
      } else if (STAGE == kCgPq && vm == 1) {
        // verification: true residual and exact stress sum of E + x
        for (int k = 0; k < nc; ++k) ss[k] = sum[1 + k];
        const double eg = e_of(sum[0]);
        publish(eg);
        G.rr[pair] = sum[0];
        if (!isfinite(eg)) st = HOM_STATUS_DIVERGED;
        else if (eg < A.tol) st = HOM_STATUS_CONVERGED;
        else if (G.steps[pair] >= A.max_iter) st = HOM_STATUS_MAX_ITER;
        else G.vmode[pair] = 2;  // restart from the true residual
      } else if (STAGE == kCgPq) {
        const double pq = sum[0];
        if (!(pq > 0.0) || !isfinite(pq)) {
          st = HOM_STATUS_DIVERGED;  // breakdown: A is not positive on this direction
        } else {
          const double alpha = G.rr[pair] / pq;
          G.alpha[pair] = alpha;
          for (int k = 0; k < nc; ++k) ss[k] += alpha * sum[1 + k];
        }
      } else if (vm == 2) {  // kCgUpdate after a failed verification: p = r
        G.beta[pair] = 0.0;
        G.vmode[pair] = 0;
      } else {  // kCgUpdate
        const double rr_new = sum[0];
        G.beta[pair] = rr_new / G.rr[pair];
        G.rr[pair] = rr_new;
        const int steps = ++G.steps[pair];
        const double eg = e_of(rr_new);
        publish(eg);
        if (!isfinite(eg)) st = HOM_STATUS_DIVERGED;
        else if (eg < A.tol) G.vmode[pair] = 1;  // verify on E + x with the next pass
        else if (steps >= A.max_iter) st = HOM_STATUS_MAX_ITER;
      }
      if (st >= 0) {
        A.status[pair] = st;
        A.iters[pair] = G.steps[pair];
        A.active[pair] = 0;
      }
    }
  }
  if (STAGE == kCgPq) return;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(A.done, 1u);
    s_last = prev == gridDim.x - 1;
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    int cnt = 0;
    for (int p = threadIdx.x; p < A.npairs; p += blockDim.x) cnt += ((volatile int*)A.active)[p] ? 1 : 0;
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    if (lane == 0) s_cnt[wid] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
      int tot = 0;
      for (int i = 0; i < (int)(blockDim.x >> 5); ++i) tot += s_cnt[i];
      *A.nactive = tot;
      *A.it_dev = it + 1;
      *A.done = 0u;
    }
  }
}

}  // namespace hom

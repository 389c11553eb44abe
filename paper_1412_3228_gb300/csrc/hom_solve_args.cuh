// Device-side arguments and reductions shared by the solver's pass kernels (generic passes in
// hom_solver.cu, the specialised 2D FP32 passes in hom_fast2d.cu).
#pragma once

#include "hom_internal.h"

namespace hom {

struct FastPlanDev;

#ifndef HOM_THREADS
#define HOM_THREADS 256
#endif
constexpr int kThreads = HOM_THREADS;  // threads per CTA of the pass kernels (a build-time tunable)
constexpr int kMaxLoads = 8;

struct SolveArgs {
  const CellDev* cells;
  const Plan* plans;
  const uint32_t* label;
  const float* mixed_c32;
  const double* mixed_c64;
  const float* phase_c32;
  const double* phase_c64;
  const double* E;  // [ncells][L][nc]
  void* eps[2];
  void* tau;
  void* g;
  double* partR;    // [ntaskR][L][nc]
  double* partC;    // [ntaskC][2]
  const TaskR* tR;
  const TaskL* tC;
  const TaskL* tY;
  const PairDev* pairs;
  int npairs;
  int* active;
  int* iters;
  int* status;
  double* err;
  double* errn;
  double* mean_sigma;  // [npairs][nc]
  double* last_err;
  int* grow;
  double* best_err;  // stagnation check: smallest error so far and its iteration
  int* best_it;
  int* it_dev;
  int* nactive;
  unsigned int* done;
  unsigned long long* bytes;  // [HOM_NKERNEL]
  int L, criterion, max_iter, diverge_window, stall_window;
  int green;  // HOM_GREEN_CONTINUOUS or HOM_GREEN_ROTATED
  int inner;  // defect-correction inner solve: the control kernel only counts iterations
  const int* kinner;  // inner solve: per-pair iteration count (the pair stops at kinner[p])
  double tol;
  void* out_eps;
  void* out_sig;
  const void* src;  // adjoint source S (nullptr for the forward solve)
  const void* src_mixed;  // defect correction: a strain added to every new iterate (mixed domain, layout of eps)
  double* res0;     // adjoint: residual sums (e, e_n) of the first iterate per pair
  const FastPlanDev* fplans;  // specialised passes: per-size tables (indexed by CellDev::fplan)
  const uint8_t* label8;      // specialised row pass: local phase index (255: mixed), x in transform order
  const int* cell_phases;     // specialised row pass: per-cell lists of the phases of pure voxels
  // whole-solve graph: the control kernel sets the WHILE condition of the graph's iteration loop
  unsigned long long cond;    // cudaGraphConditionalHandle
  int use_cond;
};

// Kahan-compensated accumulation in the field precision: the running sum s and the negated
// lost low part c (the represented value is s - c).
template <typename T> struct Acc {
  T s = T(0), c = T(0);
  __device__ __forceinline__ void add(T x) {
    T y = x - c;
    T t = s + y;
    c = (t - s) - y;
    s = t;
  }
};

// Error-free sum of (hi, lo) pairs across a warp: lane 0 ends with the total as hi + lo (TwoSum on
// the high parts, the rounding errors collected in the low parts).
template <typename T>
__device__ __forceinline__ void warp_pair_sum(T& hi, T& lo) {
  for (int o = 16; o > 0; o >>= 1) {
    const T ohi = __shfl_down_sync(0xffffffffu, hi, o);
    const T olo = __shfl_down_sync(0xffffffffu, lo, o);
    const T t = hi + ohi;
    const T bp = t - hi;
    const T err = (hi - (t - bp)) + (ohi - bp);
    hi = t;
    lo = lo + olo + err;
  }
}

// Sum K compensated partials over a block of NT threads; thread 0 gets FP64 totals in out[].
// Warps, then warp 0 over the per-warp pairs, add in the field precision with TwoSum, so FP64
// arithmetic (2 operations per SM and cycle on this GPU) is one conversion and one addition per
// total.  Every thread must call; blockDim.x must equal NT.
template <typename T, int K, int NT = kThreads>
__device__ __forceinline__ void block_sum(const Acc<T> (&v)[K], double (&out)[K]) {
  static_assert(NT % 32 == 0 && NT <= 1024, "block size");
  __shared__ T red[NT / 32][K][2];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    T hi = v[k].s, lo = -v[k].c;
    warp_pair_sum(hi, lo);
    if (lane == 0) {
      red[w][k][0] = hi;
      red[w][k][1] = lo;
    }
  }
  __syncthreads();
  if (w == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      T hi = lane < NT / 32 ? red[lane][k][0] : T(0);
      T lo = lane < NT / 32 ? red[lane][k][1] : T(0);
      warp_pair_sum(hi, lo);
      if (lane == 0) out[k] = (double)hi + (double)lo;
    }
  }
  __syncthreads();
}

// Per-cell constants of the reference medium in the field precision (precomputed on the host).
template <typename T> struct CellConst {
  T lam0, mu2, lpm, ratio, inv_mu0, inv_nv;
};
__device__ __forceinline__ void cell_const(const CellDev& c, CellConst<float>& k) {
  k = {c.f_lam0, c.f_mu2, c.f_lpm, c.f_ratio, c.f_inv_mu0, c.f_inv_nv};
}
__device__ __forceinline__ void cell_const(const CellDev& c, CellConst<double>& k) {
  k = {c.d_lam0, c.d_mu2, c.d_lpm, c.d_ratio, c.d_inv_mu0, c.d_inv_nv};
}

}  // namespace hom

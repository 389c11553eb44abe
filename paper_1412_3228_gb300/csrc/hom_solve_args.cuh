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
  // Eyre-Milton scheme: per-task sums of the compatibility residual |eps_hat - P eps_hat|^2 of the
  // Green pass, the compatibility error per pair, and (c~ + c0)^-1 of every mixed voxel (packed, in
  // the field precision, indexed like the mixed stiffness table)
  int scheme;
  double* partE;    // [ntaskC]
  double* errc;     // [npairs]
  const void* em_minv;
  // warm start: iterate 0 is the caller's field, whose g is unknown: it is neither checked nor returned
  int warm;
  // residual history: the stopping quantity of iterate i of pair p at hist[p * (max_iter + 1) + i]
  double* hist;
  // whole-solve graph: the control kernel sets the WHILE condition of the graph's iteration loop
  unsigned long long cond;    // cudaGraphConditionalHandle
  int use_cond;
  // bounds-checked builds (-DHOM_DEBUG): the first failed check's (line, file, index) and the
  // extents it is checked against (complex elements of the state and g arrays, real elements of
  // the output fields, voxels)
  unsigned int* dbg;
  size_t n_ws, n_g, n_fld, n_lab;
};

#ifndef HOM_FILE_ID
#define HOM_FILE_ID 0
#endif

// Records the first failed check (line, file, index) in w and returns false, so that the caller
// skips the access: a debug build never traps and never touches memory outside an array.
__device__ __forceinline__ bool dbg_ok(unsigned int* w, bool ok, unsigned file, unsigned line, size_t idx) {
  if (ok) return true;
  if (w && atomicCAS(w, 0u, line) == 0u) {
    w[1] = file;
    w[2] = (unsigned)(idx >> 32);
    w[3] = (unsigned)idx;
  }
  return false;
}

// Debug builds fill a pass kernel's dynamic shared memory with all-ones bytes (NaN in FP32 and
// FP64) before use, so a read of an element nobody wrote shows up as a NaN result.
__device__ __forceinline__ void dbg_poison_smem() {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned int bytes;
  asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(bytes));
  uint32_t* p = reinterpret_cast<uint32_t*>(smem_raw);
  for (unsigned i = threadIdx.x; i < bytes / 4; i += blockDim.x) p[i] = 0xFFFFFFFFu;
  __syncthreads();
}

#ifdef HOM_DEBUG
#define HOM_CHECK(A, cond, idx) ::hom::dbg_ok((A).dbg, (cond), HOM_FILE_ID, __LINE__, (size_t)(idx))
#define HOM_DBG_POISON() ::hom::dbg_poison_smem()
#else
#define HOM_CHECK(A, cond, idx) true
#define HOM_DBG_POISON() ((void)0)
#endif

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

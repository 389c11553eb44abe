// Specialised FP32 passes of the 2D fixed-point scheme (section 2, eqs. 1-a, 1-b, 2) for grid
// sizes with a compile-time radix plan.  They compute what the generic row and Green passes of
// hom_solver.cu compute, on the same mixed-domain state, task lists and partial sums; see
// hom_fast2d.cu for the data layout in shared memory.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

namespace hom {

struct SolveArgs;

// Device tables of one grid size n (plan with the radices compiled into the specialised passes).
struct FastPlanDev {
  const float4* tw4;      // (cos, cos, -sin, -sin)(2 pi t / n), t < n: twiddles duplicated per lane
  const uint16_t* iperm;  // iperm[pos]: index held at position pos after a DIF transform
  const float* xipos;     // 2 pi a(iperm[pos]): wave number of the bin at position pos
  const float* xinat;     // 2 pi a(k) in natural order
  const float2* tw2;      // the twiddle tables as (cos, -sin) pairs
  int n, pad;
};

constexpr int kFastRows = 4;  // real rows per row-pass task (two complex lines, one lane pair)
constexpr int kFastCols = 2;  // kx columns per Green-pass task (one lane pair)

// True if n has specialised 2D / 3D passes.
bool fast2d_size(int n);
bool fast3d_size(int n);
// Device tables of size n (built and uploaded on first use, kept until hom_release); every size
// of fast2d_size or fast3d_size has one.
int fast2d_plan(int n, FastPlanDev* out);
// The same tables built on the host only (no device allocation): `h` receives them and `out` their
// layout, with byte offsets from the start of `h` in place of the table pointers; after `h` is
// copied to device memory at `base`, fast2d_plan_rebase turns the offsets into device pointers.
int fast2d_plan_host(int n, std::vector<unsigned char>& h, FastPlanDev* out);
void fast2d_plan_rebase(FastPlanDev& p, const unsigned char* base);
// Dynamic shared memory of the row and Green passes for the largest grid size n of a call.
size_t fast2d_smem_row(int nmax, int nphase_cell);
size_t fast2d_smem_green(int nmax);
// Launches (one CTA per task); `smem` from fast2d_smem_row / fast2d_smem_green.
int fast2d_row(const SolveArgs& A, unsigned ntasks, size_t smem, cudaStream_t st);
int fast2d_green(const SolveArgs& A, unsigned ntasks, size_t smem, cudaStream_t st);
// Output pass (final eps and sigma fields) and the initial state eps = E, in the tiled layout of
// the specialised passes (see hom_fast2d.cu).
int fast2d_out(const SolveArgs& A, unsigned ntasks, size_t smem, cudaStream_t st);
int fast2d_init(const SolveArgs& A, int ncells, cudaStream_t st);
// label8[lp_off + y nl + pos] = index, in the cell's list of pure phases, of the phase of
// label[vox_off + y n + iperm[pos]] (255 for a mixed voxel; nl = n rounded up to 16).
int fast2d_permute_labels(const SolveArgs& A, int ncells, long long max_nv, cudaStream_t st);
void fast2d_release();

// Specialised 3D passes (hom_fast3d.cu): row, y forward / inverse, Green (z lines), the initial
// state eps = E and the output pass, on the kx-pair tiled state of those passes.
size_t fast3d_smem_row(int nmax, int nphase_cell);
size_t fast3d_smem_y(int nmax);
size_t fast3d_smem_green(int nmax);
int fast3d_row(const SolveArgs& A, unsigned ntasks, size_t smem, bool out, cudaStream_t st);
int fast3d_ypass(const SolveArgs& A, unsigned ntasks, size_t smem, bool fwd, cudaStream_t st);
int fast3d_green(const SolveArgs& A, unsigned ntasks, size_t smem, cudaStream_t st);
int fast3d_init(const SolveArgs& A, int ncells, cudaStream_t st);

}  // namespace hom

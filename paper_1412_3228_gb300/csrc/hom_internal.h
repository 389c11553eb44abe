// Host-side internals shared by the library's translation units: error reporting, the FFT
// plan cache and the device-side descriptor structs of the filter and solver kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/hom.h"
#include "hom_common.cuh"

namespace hom {

// ------------------------------------------------------------------ errors
int set_error(int code, const char* fmt, ...);
#define HOM_CUDA_TRY(call)                                                                 \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return ::hom::set_error(HOM_ERR_CUDA, "%s failed: %s (%s:%d)", #call,                \
                              cudaGetErrorString(e_), __FILE__, __LINE__);                 \
  } while (0)

// ------------------------------------------------------------------ plans
// Returns the device-resident plan of length n whose radices do not exceed max_radix (built
// and uploaded on first use), or an error.
int get_plan(int n, int max_radix, Plan* out);

// Device scratch owned by the library (grown on demand, freed by hom_release).
int get_workspace(size_t bytes, void** ptr);
void release_backward_buffers();

// ------------------------------------------------------------------ validation
bool grid_supported(int n);

// ------------------------------------------------------------------ solver body
// Caller-provided device scratch.  With a non-null base the solver places the FFT plan tables and
// all of its scratch arrays in [base, base + capacity) and makes no device allocation; a call
// that needs more than `capacity` bytes fails with HOM_ERR_UNSUPPORTED_SIZE.
struct ExternalWorkspace {
  unsigned char* base;
  size_t capacity;
};

// Adjoint Lippmann-Schwinger solve (used by hom_solve_backward): the same fixed point driven by a
// stress-sensitivity source S (real field, layout of the solver output fields) with zero mean
// strain.  The constitutive step becomes sigma' = c~ : (w - S), tau' = sigma' - c0 : w, and the
// stopping rule is relative to the residual of the first iterate (w = 0).
struct AdjointSpec {
  const void* source;  // device, [cell][load][nc][voxels] in the solve precision
};

// Validation and dispatch shared by the hom_solve entry points (ext = nullptr: library-owned
// plans and workspace; adj = nullptr: forward solve).
int solve_entry(const hom_cell* cells, int ncells, const hom_material* mat, const double* E, int L,
                const double* c0, const hom_solve_opts* opts, hom_result* out, void* stream,
                const ExternalWorkspace* ext, const AdjointSpec* adj = nullptr);

// ------------------------------------------------------------------ kernel descriptors
struct FCell {           // one cell of the filter build
  int dim, n, matrix_phase, rule, S, nprim, prim0;
  double radius_px;
  long long vox_off;
  long long block0;      // first thread block of this cell
};
struct FPrim {
  int kind, phase, axis, pad;
  double c[3];
  double radius;
};

struct CellDev {         // one cell of the solver
  int dim, n, H, Hp, nc, nrows, plan;
  long long nv;
  long long vox_off;     // voxel offset (labels)
  long long fld_off;     // element offset of the cell in the real output fields
  long long ws_off;      // complex-element offset of the cell in the mixed-domain arrays
  long long g_off;       // complex-element offset of the cell in the displacement-like array
  double lam0, mu0;
  int rtask0, rtask1;    // row-pass task range
};

struct TaskR { int cell, row0, nrows, pad; };              // rows [row0, row0+nrows) x all loads
struct TaskL { int cell, load, kx0, ntk, fixed, pad; };    // lines along one axis, kx tile

// Per (cell, load) pair
struct PairDev { int cell, load, ctask0, ctask1; };

}  // namespace hom

// Host-side internals shared by the library's translation units: error reporting, the FFT
// plan cache and the device-side descriptor structs of the filter and solver kernels.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdarg>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/hom.h"
#include "hom_common.cuh"

namespace hom {

// ------------------------------------------------------------------ tracing
// NVTX range for the lifetime of the object (entry points, solve phases, pass launches); costs a
// few nanoseconds when no profiler is attached.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { end(); }
  void end() {  // close early (once); the destructor closes it on every other path
    if (open_) nvtxRangePop();
    open_ = false;
  }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;

 private:
  bool open_ = true;
};

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

// Points a plan's table pointers into device memory laid out by fill_plan_tables.
inline void set_plan_pointers(Plan& p, unsigned char* base) {
  auto up = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t n = (size_t)p.n;
  p.perm = reinterpret_cast<const uint16_t*>(base);
  base += up(n * 2);
  p.tw32 = reinterpret_cast<const float2*>(base);
  base += up(n * 8);
  p.tw64 = reinterpret_cast<const double2*>(base);
  base += up(n * 16);
  p.xi32 = reinterpret_cast<const float*>(base);
  base += up(n * 4);
  p.xi64 = reinterpret_cast<const double*>(base);
  base += up(n * 8);
  p.rot32 = reinterpret_cast<const float2*>(base);
  base += up(n * 8);
  p.rot64 = reinterpret_cast<const double2*>(base);
}

// Device scratch owned by the library (grown on demand, freed by hom_release).
int get_workspace(size_t bytes, void** ptr);
void release_backward_buffers();
void release_graphs();  // cached whole-solve graphs
std::string tune_report();  // the autotuner's choices and timings, one line per batch shape

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
                const ExternalWorkspace* ext, const AdjointSpec* adj = nullptr, bool cg = false);

// ------------------------------------------------------------------ kernel descriptors
struct FCell {           // one cell of the filter build
  int dim, n, matrix_phase, rule, S, nprim, prim0;
  double radius_px;
  long long vox_off;
  long long block0;      // first thread block of this cell
  float inv_n;           // 1 / n rounded to FP32
  float reach32;         // filter radius in cell units (r / n) rounded to FP32
  int R2i;               // (2 S r)^2 rounded down: a fine point is in the ball iff sum D^2 <= R2i
  int tlo, thi;          // range of the fine-point offsets t that can fall in a ball
  int M;                 // fine points per ball
  FastDiv dn, dnt;       // dividers by n and by thi - tlo + 1
};
struct FPrim {
  int kind, phase, axis, pad;
  double c[3];
  double radius;
  float c32[3], r32;     // centre and radius (slab: thickness) rounded to FP32
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
  int fplan;             // specialised passes: index of the size's tables (-1: generic passes)
  long long lp_off;      // specialised passes: byte offset of the cell in the one-byte labels (16-aligned)
  int ph_off, nph;       // specialised passes: the cell's pure phases, cell_phases[ph_off .. ph_off + nph)
  // per-cell constants, computed on the host (FP64 arithmetic is slow on the device)
  float f_lam0, f_mu2, f_lpm, f_ratio, f_inv_mu0, f_inv_nv;
  double d_lam0, d_mu2, d_lpm, d_ratio, d_inv_mu0, d_inv_nv;
};

struct TaskR { int cell, row0, nrows, load; };  // rows [row0, row0+nrows) x one load (load < 0: every load)
struct TaskL {  // lines along one axis for a tile of kx: ntk columns x nc components
  int cell, load, kx0, ntk, fixed, pad;
  FastDiv d_ntk, d_nl, d_ng;  // dividers by ntk, ntk * nc and ntk * dim
};

// Per (cell, load) pair
struct PairDev { int cell, load, ctask0, ctask1, rtask0, rtask1; };  // Green- and row-pass task ranges

}  // namespace hom

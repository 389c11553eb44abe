// hom_solve_noalloc: the fixed-point solve for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc: a framework may have reserved the device memory up front
// for its own caching allocator (so a foreign cudaMalloc fails or fragments its pool), a service
// may run under a hard per-process memory budget, and cudaFree synchronises the whole device,
// which latency-sensitive callers cannot afford.  This entry point runs the same kernels as
// hom_solve (the specialised FP32 passes included) but takes all of its scratch -- the FFT plan
// tables, the mixed-domain state, the partial sums and the convergence bookkeeping -- from one
// array of fixed size that lives in the library's device memory.  The caller still owns and
// passes every input and output buffer.
#include "hom_internal.h"

namespace {

// Largest solver scratch a hom_solve_noalloc call may use (64 MiB).  Every device that loads the
// library keeps this array until the process exits.
constexpr size_t kNoAllocScratchBytes = size_t(64) << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of the array in the current context.  In host code the array's name only stands
// for it; the real address comes from cudaGetSymbolAddress with the device current.  It is looked
// up on every call (a cheap query once the module is loaded), so a context re-created after
// cudaDeviceReset, or another context made current, never sees a stale address.
int scratch_address(void** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || p == nullptr)
    return hom::set_error(HOM_ERR_CUDA, "hom_solve_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
  *out = p;
  return HOM_OK;
}

}  // namespace

extern "C" int hom_solve_noalloc(const hom_cell* cells, int32_t ncells, const hom_material* mat, const double* E,
                                 int32_t L, const double* c0, const hom_solve_opts* opts, hom_result* out,
                                 void* stream) {
  ::hom::NvtxRange nvtx_range_("hom_solve_noalloc");
  cudaGetLastError();  // do not report an error left behind by an unrelated earlier call
  if (!opts || !out)
    return hom::set_error(HOM_ERR_INVALID_ARG, "hom_solve_noalloc: null argument");
  if (opts->use_graph)
    return hom::set_error(HOM_ERR_INVALID_ARG, "hom_solve_noalloc: use_graph must be 0 (graphs allocate)");
  if (out->stats)
    return hom::set_error(HOM_ERR_INVALID_ARG, "hom_solve_noalloc: stats must be NULL (timing events allocate)");
  void* base = nullptr;
  int rc = scratch_address(&base);
  if (rc != HOM_OK) return rc;
  const hom::ExternalWorkspace ext{static_cast<unsigned char*>(base), kNoAllocScratchBytes};
  rc = hom::solve_entry(cells, ncells, mat, E, L, c0, opts, out, stream, &ext);
  if (rc != HOM_OK && rc != HOM_ERR_NOT_CONVERGED && rc != HOM_ERR_DIVERGED) {
    // A failure may come after kernels were queued on the stream: wait for them, so that a caller
    // who takes the return as completion does not start another call on the shared array while
    // this one still runs (the wait's own status is not reported; the first error is).
    cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  }
  return rc;
}

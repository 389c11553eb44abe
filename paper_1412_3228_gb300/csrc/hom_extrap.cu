// Fourier extrapolation of the filtered stiffness (section 6, Fig. 4): one component of c~(x_a) is
// expanded in the truncated Fourier series whose coefficients are the DFT of its grid values on the
// odd frequency set J, and the series is evaluated at the voxel centres of a finer m^dim grid.
//
// The series f(y) = n^-dim sum_{k in J} c_hat(k) exp(2 pi i k.(y - x_0)) is evaluated in its
// equivalent real form, the separable Dirichlet-kernel sum
//     f(y) = sum_a c(x_a) prod_d D_n(y_d - x_{a,d}),   D_n(t) = n^-1 sum_{k in J} e^{2 pi i k t},
// one axis at a time: x first (n^(dim-1) rows of length n -> m), then y, then z.  Every step is a
// short FP64 dot product of length n per output point; the whole call costs n m^dim (1 + n/m + ...)
// multiply-adds, a few milliseconds for the 3D sizes it is meant for, so the kernels are plain
// one-output-per-thread loops.
#include "hom_internal.h"

namespace hom {
namespace {

constexpr int kT = 256;

// D[a][b] = D_n(y_b - x_a) with x_a = (a + 1/2)/n, y_b = (b + 1/2)/m.  The argument is
// t = q / (2 m n) with the exact integer q = (2b + 1) n - (2a + 1) m; D_n has period 1 for odd n,
// so q is reduced modulo 2 m n, and q = 0 (y_b = x_a) gives D_n = 1.  Otherwise
// D_n(t) = sin(n pi t) / (n sin(pi t)) with 0 < t < 1.
__global__ void k_dirichlet(double* __restrict__ D, int n, int m) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)n * m) return;
  const int a = (int)(idx / m), b = (int)(idx % m);
  const int64_t P = 2LL * m * n;
  int64_t q = ((int64_t)(2 * b + 1) * n - (int64_t)(2 * a + 1) * m) % P;
  if (q < 0) q += P;
  D[idx] = q == 0 ? 1.0 : sinpi((double)q / (2.0 * m)) / ((double)n * sinpi((double)q / (double)P));
}

// v[i] = packed component `comp` of c~ at voxel i of the cell (labels of one cell).
__global__ void k_component(const uint32_t* __restrict__ label, int64_t nv, const double* __restrict__ phase_c,
                            const double* __restrict__ mixed_c, int ns, int comp, double* __restrict__ v) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nv) return;
  const uint32_t l = label[i];
  v[i] = (l & HOM_MIXED_BIT) ? mixed_c[(int64_t)(l & ~HOM_MIXED_BIT) * ns + comp] : phase_c[(int64_t)l * ns + comp];
}

// out[o][b][i] = sum_a D[a][b] in[o][a][i]: the series summed along one axis of an [O][n][I] array.
// Consecutive threads take consecutive i (coalesced rows when I > 1) or consecutive b (I == 1).
__global__ void k_axis(const double* __restrict__ in, double* __restrict__ out, const double* __restrict__ D,
                       int64_t O, int n, int m, int64_t I) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= O * m * I) return;
  const int64_t i = idx % I;
  const int64_t r = idx / I;
  const int b = (int)(r % m);
  const int64_t o = r / m;
  const double* src = in + o * n * I + i;
  double s = 0.0;
  for (int a = 0; a < n; ++a) s = fma(D[(int64_t)a * m + b], src[(int64_t)a * I], s);
  out[idx] = s;
}

bool on_device(const void* p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

unsigned blocks_for(int64_t count) { return (unsigned)((count + kT - 1) / kT); }

}  // namespace
}  // namespace hom

extern "C" int hom_fourier_extrapolate(const hom_cell* cells, int32_t ncells, const hom_material* mat, int32_t cell,
                                       int32_t comp, int32_t m, double* out, void* stream) {
  ::hom::NvtxRange nvtx_range_("hom_fourier_extrapolate");
  using namespace hom;
  if (!cells || ncells <= 0 || !mat || !mat->label || !mat->phase_c64 || !out)
    return set_error(HOM_ERR_INVALID_ARG, "hom_fourier_extrapolate: null or empty argument");
  if (cell < 0 || cell >= ncells)
    return set_error(HOM_ERR_INVALID_ARG, "hom_fourier_extrapolate: cell %d out of range [0, %d)", cell, ncells);
  const int dim = cells[0].dim;
  if ((dim != 2 && dim != 3) || mat->dim != dim)
    return set_error(HOM_ERR_INVALID_ARG, "hom_fourier_extrapolate: dim %d does not match the material", dim);
  int64_t off = 0;
  for (int c = 0; c < ncells; ++c) {
    if (cells[c].dim != dim) return set_error(HOM_ERR_INVALID_ARG, "cell %d: every cell must share dim %d", c, dim);
    if (c < cell) off += dim == 2 ? (int64_t)cells[c].n * cells[c].n : (int64_t)cells[c].n * cells[c].n * cells[c].n;
  }
  const int n = cells[cell].n;
  if (!grid_supported(n) || (n & 1) == 0)  // J is symmetric (a real series) for odd grids only
    return set_error(HOM_ERR_UNSUPPORTED_SIZE, "cell %d: grid %d is not an odd supported size", cell, n);
  const int ns = dim == 2 ? 6 : 21;
  if (comp < 0 || comp >= ns)
    return set_error(HOM_ERR_INVALID_ARG, "hom_fourier_extrapolate: component %d out of range [0, %d)", comp, ns);
  if (m < 1 || (dim == 3 && m > 1024) || (dim == 2 && m > 32768))
    return set_error(HOM_ERR_INVALID_ARG, "hom_fourier_extrapolate: fine grid %d out of range", m);
  if (mat->mixed_count > 0 && !mat->mixed_c64)
    return set_error(HOM_ERR_INVALID_ARG, "hom_fourier_extrapolate: mixed table missing");

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t nv = dim == 2 ? (int64_t)n * n : (int64_t)n * n * n;
  const int64_t mm = (int64_t)m * m;
  const int64_t nout = dim == 2 ? mm : mm * m;
  const bool dev_out = on_device(out);
  // scratch: grid values, D, the partial sums after each axis but the last, and a device copy of
  // the result when `out` is host memory
  const int64_t sizes[5] = {nv, (int64_t)n * m, dim == 2 ? (int64_t)n * m : (int64_t)n * n * m,
                            dim == 2 ? 0 : (int64_t)n * mm, dev_out ? 0 : nout};
  double* buf[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  int rc = HOM_OK;
  for (int i = 0; i < 5 && rc == HOM_OK; ++i) {
    if (!sizes[i]) continue;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&buf[i]), sizes[i] * sizeof(double), s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      buf[i] = nullptr;
      rc = set_error(HOM_ERR_OOM, "hom_fourier_extrapolate: scratch of %lld bytes: %s",
                     (long long)(sizes[i] * sizeof(double)), cudaGetErrorString(e));
    }
  }
  if (rc == HOM_OK) {
    double* v = buf[0];
    double* D = buf[1];
    double* dst = dev_out ? out : buf[4];
    k_component<<<blocks_for(nv), kT, 0, s>>>(mat->label + off, nv, mat->phase_c64, mat->mixed_c64, ns, comp, v);
    k_dirichlet<<<blocks_for((int64_t)n * m), kT, 0, s>>>(D, n, m);
    if (dim == 2) {
      k_axis<<<blocks_for((int64_t)n * m), kT, 0, s>>>(v, buf[2], D, n, n, m, 1);       // x: [y][x] -> [y][bx]
      k_axis<<<blocks_for(mm), kT, 0, s>>>(buf[2], dst, D, 1, n, m, m);                 // y: -> [by][bx]
    } else {
      k_axis<<<blocks_for((int64_t)n * n * m), kT, 0, s>>>(v, buf[2], D, (int64_t)n * n, n, m, 1);  // x
      k_axis<<<blocks_for((int64_t)n * mm), kT, 0, s>>>(buf[2], buf[3], D, n, n, m, m);              // y
      k_axis<<<blocks_for(nout), kT, 0, s>>>(buf[3], dst, D, 1, n, m, mm);                           // z
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) rc = set_error(HOM_ERR_CUDA, "hom_fourier_extrapolate: launch failed: %s", cudaGetErrorString(e));
    if (rc == HOM_OK && !dev_out) {
      e = cudaMemcpyAsync(out, dst, nout * sizeof(double), cudaMemcpyDeviceToHost, s);
      if (e != cudaSuccess) rc = set_error(HOM_ERR_CUDA, "hom_fourier_extrapolate: copy failed: %s", cudaGetErrorString(e));
    }
  }
  for (int i = 0; i < 5; ++i)
    if (buf[i]) cudaFreeAsync(buf[i], s);
  cudaError_t e = cudaStreamSynchronize(s);
  if (rc == HOM_OK && e != cudaSuccess)
    rc = set_error(HOM_ERR_CUDA, "hom_fourier_extrapolate: %s", cudaGetErrorString(e));
  return rc;
}

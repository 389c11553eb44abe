// hom_solve_backward: reverse-mode derivative of a loss L(C_eff, sigma fields) through the basic
// scheme of section 2 (eqs. 1-a, 1-b, 2) and the filter rules (eqs. 3, 4, 5-a, 5-b).
//
// With the converged fields eps^(j) of the nc unit Mandel loads, C_ij = <eps^(i) : c~ : eps^(j)>
// holds exactly at the discrete solution (the projection onto compatible fields is orthogonal: on
// odd grids, and on even grids with the Nyquist wave vectors set to zero strain), so
//   dC_ij / dc~(x) = eps^(i)(x) (x) eps^(j)(x) / N_v.
// For J = sum_j sum_x S^(j)(x) . sigma^(j)(x) with S^(j) = dL/dsigma^(j), the adjoint field
// w^(j) (compatible, zero mean) solves the same Lippmann-Schwinger fixed point with source c~ S:
//   w = -Gamma0 * ((c~ - c0) : w - c~ : S),   w_hat(0) = 0,
// and dJ / dc~(x) = sum_j (S^(j)(x) - w^(j)(x)) (x) eps^(j)(x).
// Gradients with respect to the phase Lame constants and to the volume fractions of mixed voxels
// follow from the chain rule through each voxel's rule, evaluated in forward mode (dual numbers).
#include <cstring>
#include <vector>

#include "hom_internal.h"
#include "hom_rules.cuh"

namespace hom {
namespace {

constexpr int kThreads = 128;
constexpr int kMaxSlots = 4;  // distinct phases referenced by one cell

struct GCell {
  int dim, n, rule, nslot;
  int slot_phase[kMaxSlots];
  long long vox_off, fld_off, nv, block0;
};

struct GradArgs {
  const GCell* cells;
  int ncells, L;
  const uint32_t* label;
  const int32_t* mixed_phases;
  const double* mixed_frac;
  const double* mixed_normal;
  const double* phase_lame;  // [nphase][2]
  const double* dLdC;        // [ncells][nc][nc] or nullptr
  const void* eps;           // forward strain fields
  const void* S;             // dL/dsigma fields or nullptr
  const void* w;             // adjoint fields or nullptr
  void* dctilde;             // [sum voxels][ns] or nullptr
  double* dfrac;             // [mixed capacity] or nullptr
  double* dphase;            // [nphase][2]
};

template <typename T, int DIM>
__global__ void __launch_bounds__(kThreads) k_grad(GradArgs A) {
  constexpr int NC = DIM == 2 ? 3 : 6;
  constexpr int NS = DIM == 2 ? 6 : 21;
  int ci = 0;
  for (int c = 1; c < A.ncells; ++c)
    if ((long long)blockIdx.x >= A.cells[c].block0) ci = c;
  const GCell cell = A.cells[ci];
  const long long v = ((long long)blockIdx.x - cell.block0) * kThreads + threadIdx.x;
  double contrib[kMaxSlots][2];
  for (int s = 0; s < kMaxSlots; ++s) contrib[s][0] = contrib[s][1] = 0.0;
  if (v < cell.nv) {
    const int L = A.L;
    const T* eps = static_cast<const T*>(A.eps) + cell.fld_off + v;
    // gradient with respect to the full Mandel matrix c~_pq, accumulated in the field precision
    T Am[NC][NC];
#pragma unroll
    for (int p = 0; p < NC; ++p)
#pragma unroll
      for (int q = 0; q < NC; ++q) Am[p][q] = T(0);
    // C_eff term: (1/N_v) sum_ij G_ij eps^(i)_p eps^(j)_q (loads are the nc unit strains)
    if (A.dLdC) {
      const double* G = A.dLdC + (size_t)ci * NC * NC;
      const T inv_nv = (T)(1.0 / (double)cell.nv);
      for (int i = 0; i < NC; ++i) {
        T u[NC];
#pragma unroll
        for (int q = 0; q < NC; ++q) u[q] = T(0);
        for (int j = 0; j < NC; ++j) {
          const T g = (T)G[i * NC + j];
          if (g == T(0)) continue;
#pragma unroll
          for (int q = 0; q < NC; ++q) u[q] += g * eps[((size_t)j * NC + q) * cell.nv];
        }
#pragma unroll
        for (int p = 0; p < NC; ++p) {
          const T ep = eps[((size_t)i * NC + p) * cell.nv] * inv_nv;
#pragma unroll
          for (int q = 0; q < NC; ++q) Am[p][q] += ep * u[q];
        }
      }
    }
    // local stress term: sum_j (S^(j) - w^(j))_p eps^(j)_q
    if (A.S) {
      const T* S = static_cast<const T*>(A.S) + cell.fld_off + v;
      const T* W = A.w ? static_cast<const T*>(A.w) + cell.fld_off + v : nullptr;
      for (int j = 0; j < L; ++j) {
        T d[NC], e[NC];
#pragma unroll
        for (int k = 0; k < NC; ++k) {
          const size_t o = ((size_t)j * NC + k) * cell.nv;
          d[k] = S[o] - (W ? W[o] : T(0));
          e[k] = eps[o];
        }
#pragma unroll
        for (int p = 0; p < NC; ++p)
#pragma unroll
          for (int q = 0; q < NC; ++q) Am[p][q] += d[p] * e[q];
      }
    }
    // packed gradient: entry (p <= q) moves both c~_pq and c~_qp
    if (A.dctilde) {
      T* out = static_cast<T*>(A.dctilde) + (size_t)(cell.vox_off + v) * NS;
#pragma unroll
      for (int p = 0; p < NC; ++p)
#pragma unroll
        for (int q = p; q < NC; ++q) out[packed_index(NC, p, q)] = (T)(p == q ? Am[p][p] : Am[p][q] + Am[q][p]);
    }
    const uint32_t lab = A.label[cell.vox_off + v];
    if (!(lab & HOM_MIXED_BIT)) {
      // pure voxel: c = lam 1(x)1 + 2 mu I  ->  dL/dlam = sum over the normal block, dL/dmu = 2 tr
      T dl = T(0), dm = T(0);
#pragma unroll
      for (int p = 0; p < DIM; ++p)
#pragma unroll
        for (int q = 0; q < DIM; ++q) dl += Am[p][q];
#pragma unroll
      for (int p = 0; p < NC; ++p) dm += T(2) * Am[p][p];
      for (int s = 0; s < cell.nslot; ++s)
        if (cell.slot_phase[s] == (int)lab) { contrib[s][0] += dl; contrib[s][1] += dm; }
    } else {
      // mixed voxel: directional derivatives of the rule by dual numbers
      const uint32_t m = lab & ~HOM_MIXED_BIT;
      const int pa = A.mixed_phases[2 * m], pb = A.mixed_phases[2 * m + 1];
      const double fb = A.mixed_frac[m];
      double nrm[3] = {A.mixed_normal[3 * m], A.mixed_normal[3 * m + 1], A.mixed_normal[3 * m + 2]};
      const bool nrm_ok = (nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2]) > 0.25;
      const double lam[2] = {A.phase_lame[2 * pa], A.phase_lame[2 * pb]};
      const double mu[2] = {A.phase_lame[2 * pa + 1], A.phase_lame[2 * pb + 1]};
      double dtheta[5];
      for (int dir = 0; dir < 5; ++dir) {  // lam_a, mu_a, lam_b, mu_b, f_b
        Dual Cs[2][36], fs[2], Ct[36];
        for (int k = 0; k < 2; ++k) {
          const Dual l = {lam[k], (dir == 2 * k) ? 1.0 : 0.0};
          const Dual u = {mu[k], (dir == 2 * k + 1) ? 1.0 : 0.0};
          iso_full_t<Dual>(l, u, DIM, Cs[k]);
        }
        fs[1] = {fb, dir == 4 ? 1.0 : 0.0};
        fs[0] = {1.0 - fb, dir == 4 ? -1.0 : 0.0};
        apply_rule_t<Dual>(cell.rule, 2, Cs, fs, nrm_ok, nrm, DIM, Ct);
        double s = 0.0;
#pragma unroll
        for (int p = 0; p < NC; ++p)
#pragma unroll
          for (int q = 0; q < NC; ++q) s += (double)Am[p][q] * Ct[p * NC + q].d;
        dtheta[dir] = s;
      }
      for (int s = 0; s < cell.nslot; ++s) {
        if (cell.slot_phase[s] == pa) { contrib[s][0] += dtheta[0]; contrib[s][1] += dtheta[1]; }
        if (cell.slot_phase[s] == pb) { contrib[s][0] += dtheta[2]; contrib[s][1] += dtheta[3]; }
      }
      if (A.dfrac) A.dfrac[m] = dtheta[4];
    }
  }
  // block reduction of the phase contributions, one atomic per block and slot
  __shared__ double red[kThreads / 32][kMaxSlots][2];
  const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
  for (int s = 0; s < kMaxSlots; ++s)
    for (int k = 0; k < 2; ++k) {
      double x = contrib[s][k];
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      if (lane == 0) red[wq][s][k] = x;
    }
  __syncthreads();
  if (threadIdx.x < cell.nslot * 2) {
    const int s = threadIdx.x >> 1, k = threadIdx.x & 1;
    double t = 0.0;
    for (int i = 0; i < kThreads / 32; ++i) t += red[i][s][k];
    atomicAdd(A.dphase + 2 * cell.slot_phase[s] + k, t);
  }
}

struct AuxCache {
  void* p = nullptr;
  size_t bytes = 0;
};
AuxCache g_aux[64];  // per device: the adjoint fields w (freed by hom_release)

int aux_buffer(size_t bytes, void** out) {
  int dev = 0;
  HOM_CUDA_TRY(cudaGetDevice(&dev));
  AuxCache& a = g_aux[dev & 63];
  if (bytes > a.bytes) {
    if (a.p) {
      cudaDeviceSynchronize();
      cudaFree(a.p);
    }
    a.p = nullptr;
    a.bytes = 0;
    const cudaError_t e = cudaMalloc(&a.p, bytes);
    if (e != cudaSuccess) return set_error(HOM_ERR_OOM, "backward buffer of %zu bytes: %s", bytes, cudaGetErrorString(e));
    a.bytes = bytes;
  }
  *out = a.p;
  return HOM_OK;
}

}  // namespace

void release_backward_buffers() {
  for (int d = 0; d < 64; ++d)
    if (g_aux[d].p) {
      cudaSetDevice(d);
      cudaDeviceSynchronize();
      cudaFree(g_aux[d].p);
      g_aux[d].p = nullptr;
      g_aux[d].bytes = 0;
    }
}

}  // namespace hom

using namespace hom;

extern "C" int hom_solve_backward(const hom_cell* cells, int32_t ncells, const hom_material* mat, const double* c0,
                                  int32_t L, const hom_solve_opts* opts, const void* eps, const double* dL_dC,
                                  const void* dL_dsigma, void* dL_dctilde, double* dL_dphase, double* dL_dfrac,
                                  hom_result* adjoint_info, void* stream) {
  ::hom::NvtxRange nvtx_range_("hom_solve_backward");
  cudaGetLastError();  // do not report an error left behind by an unrelated earlier call
  if (!cells || ncells <= 0 || !mat || !c0 || !opts || !eps || !dL_dphase)
    return set_error(HOM_ERR_INVALID_ARG, "hom_solve_backward: null argument");
  if (!dL_dC && !dL_dsigma) return set_error(HOM_ERR_INVALID_ARG, "hom_solve_backward: no loss gradient given");
  const int dim = cells[0].dim;
  const int nc = nc_of(dim);
  if (dL_dC && L != nc)
    return set_error(HOM_ERR_INVALID_ARG, "hom_solve_backward: dL_dC needs the %d unit Mandel load cases", nc);
  if (L < 1 || L > 8) return set_error(HOM_ERR_INVALID_ARG, "hom_solve_backward: L out of range");
  if (mat->dim != dim) return set_error(HOM_ERR_INVALID_ARG, "hom_solve_backward: material dimension mismatch");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t tsize = opts->precision == HOM_FP32 ? sizeof(float) : sizeof(double);
  size_t nfield = 0, nvox = 0;
  for (int c = 0; c < ncells; ++c) {
    const size_t nv = (size_t)cells[c].n * cells[c].n * (dim == 3 ? cells[c].n : 1);
    nfield += (size_t)L * nc * nv;
    nvox += nv;
  }
  // 1. adjoint solve (only with a local-stress term)
  void* w = nullptr;
  int adj_code = HOM_OK;
  if (dL_dsigma) {
    int rc = aux_buffer(nfield * tsize, &w);
    if (rc != HOM_OK) return rc;
    std::vector<double> zeroE((size_t)ncells * L * nc, 0.0), msig((size_t)ncells * L * nc);
    hom_result r{};
    r.eps = w;
    r.mean_sigma = msig.data();
    if (adjoint_info) {
      r.iterations = adjoint_info->iterations;
      r.status = adjoint_info->status;
      r.err = adjoint_info->err;
      r.err_n = adjoint_info->err_n;
    }
    AdjointSpec adj{dL_dsigma};
    adj_code = solve_entry(cells, ncells, mat, zeroE.data(), L, c0, opts, &r, stream, nullptr, &adj);
    if (adj_code != HOM_OK && adj_code != HOM_ERR_NOT_CONVERGED) return adj_code;
  }
  // 2. gradient assembly
  std::vector<GCell> gc(ncells);
  long long blocks = 0, vox = 0, fld = 0;
  for (int c = 0; c < ncells; ++c) {
    const hom_cell& k = cells[c];
    GCell& g = gc[c];
    g.dim = dim;
    g.n = k.n;
    g.rule = k.rule;
    g.nv = (long long)k.n * k.n * (dim == 3 ? k.n : 1);
    g.vox_off = vox;
    g.fld_off = fld;
    g.block0 = blocks;
    g.nslot = 0;
    auto add_slot = [&](int ph) {
      for (int s = 0; s < g.nslot; ++s)
        if (g.slot_phase[s] == ph) return true;
      if (g.nslot == kMaxSlots) return false;
      g.slot_phase[g.nslot++] = ph;
      return true;
    };
    bool ok = add_slot(k.matrix_phase);
    for (int p = 0; p < k.nprim; ++p) ok = ok && add_slot(k.prims[p].phase);
    if (!ok) return set_error(HOM_ERR_INVALID_ARG, "hom_solve_backward: cell %d references more than %d phases", c, kMaxSlots);
    vox += g.nv;
    fld += (long long)L * nc * g.nv;
    blocks += (g.nv + kThreads - 1) / kThreads;
  }
  const int nphase = mat->nphase;
  std::vector<double> lame(2 * (size_t)nphase);
  {
    // recover the Lame constants from the packed phase table (c_00 = lam + 2 mu, c_01 = lam)
    std::vector<double> pc((size_t)nphase * ns_of(dim));
    HOM_CUDA_TRY(cudaMemcpyAsync(pc.data(), mat->phase_c64, pc.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    HOM_CUDA_TRY(cudaStreamSynchronize(st));
    for (int p = 0; p < nphase; ++p) {
      const double* q = pc.data() + (size_t)p * ns_of(dim);
      lame[2 * p] = q[packed_index(nc, 0, 1)];
      lame[2 * p + 1] = 0.5 * (q[packed_index(nc, 0, 0)] - q[packed_index(nc, 0, 1)]);
    }
  }
  const size_t b_cells = (sizeof(GCell) * ncells + 255) / 256 * 256;
  const size_t b_lame = (sizeof(double) * lame.size() + 255) / 256 * 256;
  const size_t b_G = dL_dC ? ((sizeof(double) * ncells * nc * nc + 255) / 256 * 256) : 0;
  const size_t b_ph = (sizeof(double) * 2 * nphase + 255) / 256 * 256;
  void* ws = nullptr;
  int rc = get_workspace(b_cells + b_lame + b_G + b_ph, &ws);
  if (rc != HOM_OK) return rc;
  unsigned char* wb = static_cast<unsigned char*>(ws);
  HOM_CUDA_TRY(cudaMemcpyAsync(wb, gc.data(), sizeof(GCell) * ncells, cudaMemcpyHostToDevice, st));
  HOM_CUDA_TRY(cudaMemcpyAsync(wb + b_cells, lame.data(), sizeof(double) * lame.size(), cudaMemcpyHostToDevice, st));
  if (dL_dC)
    HOM_CUDA_TRY(cudaMemcpyAsync(wb + b_cells + b_lame, dL_dC, sizeof(double) * ncells * nc * nc,
                                 cudaMemcpyHostToDevice, st));
  double* dph = reinterpret_cast<double*>(wb + b_cells + b_lame + b_G);
  HOM_CUDA_TRY(cudaMemsetAsync(dph, 0, sizeof(double) * 2 * nphase, st));
  GradArgs A{};
  A.cells = reinterpret_cast<const GCell*>(wb);
  A.ncells = ncells;
  A.L = L;
  A.label = mat->label;
  A.mixed_phases = mat->mixed_phases;
  A.mixed_frac = mat->mixed_frac;
  A.mixed_normal = mat->mixed_normal;
  A.phase_lame = reinterpret_cast<const double*>(wb + b_cells);
  A.dLdC = dL_dC ? reinterpret_cast<const double*>(wb + b_cells + b_lame) : nullptr;
  A.eps = eps;
  A.S = dL_dsigma;
  A.w = w;
  A.dctilde = dL_dctilde;
  A.dfrac = dL_dfrac;
  A.dphase = dph;
  if (opts->precision == HOM_FP32) {
    if (dim == 2) k_grad<float, 2><<<(unsigned)blocks, kThreads, 0, st>>>(A);
    else k_grad<float, 3><<<(unsigned)blocks, kThreads, 0, st>>>(A);
  } else {
    if (dim == 2) k_grad<double, 2><<<(unsigned)blocks, kThreads, 0, st>>>(A);
    else k_grad<double, 3><<<(unsigned)blocks, kThreads, 0, st>>>(A);
  }
  HOM_CUDA_TRY(cudaGetLastError());
  HOM_CUDA_TRY(cudaMemcpyAsync(dL_dphase, dph, sizeof(double) * 2 * nphase, cudaMemcpyDeviceToHost, st));
  HOM_CUDA_TRY(cudaStreamSynchronize(st));
  (void)nvox;
  if (adj_code == HOM_ERR_NOT_CONVERGED) set_error(adj_code, "adjoint solve reached max_iter");
  return adj_code;
}

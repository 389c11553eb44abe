// Filtered stiffness c~(x_a) = HR(c, w(x_a)) of section 2 (eqs. 3, 4, 5-a, 5-b): one thread per
// voxel.  The thread classifies the voxel with analytic distances to the primitive surfaces;
// only voxels whose filter ball can reach a surface count fine-grid samples per phase, and
// only voxels whose samples hold two phases get a mixed-table entry with the rule applied.
//
// Exactness.  Sample coordinates are integers in units of h/(2S) (sample 2j+1, voxel centre
// (2a+1)S), the ball test sum D^2 <= (2 S r)^2 compares an exact integer, and the membership
// test of a sample in a primitive is a fixed sequence of IEEE FP64 operations written with
// explicit round-to-nearest intrinsics (no contraction into fused multiply-adds), so the counts
// equal those of any implementation performing the same operations.
#include <cstdio>
#include <cstring>
#include <vector>

#include "hom_internal.h"
#include "hom_rules.cuh"

namespace hom {
namespace {

constexpr int kThreads = 128;
constexpr int kMaxNear = 8;     // primitives whose surface can cross one ball
constexpr int kMaxPhases = 4;   // distinct phases inside one ball

__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }

// Exact membership of a sample (u-unit coordinates su[0..dim)) in primitive p:
//   cu = c * (2 S n); du = su - cu; wrap du by +-2 S n into [-S n, S n];
//   disk/sphere: ((du_x^2 + du_y^2) + du_z^2) <= (R * 2 S n)^2;  slab: |du_axis| <= T * (S n)
__device__ bool inside_exact(const FPrim& p, const double* su, int dim, double P2, double half) {
  auto wrapped = [&](int ax) {
    double du = dsub(su[ax], dmul(p.c[ax], P2));
    if (du > half) du = dsub(du, P2);
    if (du < -half) du = dadd(du, P2);
    return du;
  };
  if (p.kind == HOM_PRIM_SLAB) {
    double du = wrapped(p.axis);
    return fabs(du) <= dmul(p.radius, half);
  }
  const double Ru = dmul(p.radius, P2);
  const double Ru2 = dmul(Ru, Ru);
  double w = wrapped(0);
  double q = dmul(w, w);
  for (int ax = 1; ax < dim; ++ax) {
    w = wrapped(ax);
    q = dadd(q, dmul(w, w));
  }
  return q <= Ru2;
}

struct FilterArgs {
  const FCell* cells;
  int ncells;
  const FPrim* prims;
  const double* phase_lame;  // [nphase][2]
  int nphase;
  hom_material mat;
  unsigned long long* mixed_counter;
  int* err_flag;             // 1: 2-layer with more than two phases, 2: too many phases/primitives
};

__global__ void __launch_bounds__(kThreads) k_filter(FilterArgs A) {
  // locate the cell of this block (cells are few: linear search)
  int ci = 0;
  for (int c = 1; c < A.ncells; ++c)
    if ((long long)blockIdx.x >= A.cells[c].block0) ci = c;
  const FCell cell = A.cells[ci];
  const long long nv = (long long)cell.n * cell.n * (cell.dim == 3 ? cell.n : 1);
  const long long v = ((long long)blockIdx.x - cell.block0) * kThreads + threadIdx.x;
  if (v >= nv) return;
  const int n = cell.n, dim = cell.dim, S = cell.S;
  int a[3] = {(int)(v % n), (int)((v / n) % n), dim == 3 ? (int)(v / ((long long)n * n)) : 0};
  const double P2 = 2.0 * (double)S * (double)n;
  const double half = (double)S * (double)n;
  const FPrim* prims = A.prims + cell.prim0;

  // phase of the grid point itself (exact recipe)
  double sc[3];
  for (int d = 0; d < dim; ++d) sc[d] = (double)(2 * a[d] + 1) * (double)S;
  int centre_first = -1;  // first primitive containing the centre
  for (int p = 0; p < cell.nprim; ++p)
    if (inside_exact(prims[p], sc, dim, P2, half)) { centre_first = p; break; }
  const int centre_phase = centre_first >= 0 ? prims[centre_first].phase : cell.matrix_phase;
  uint32_t* label = A.mat.label + cell.vox_off + v;
  if (cell.rule == HOM_RULE_NONE || cell.nprim == 0) {
    *label = (uint32_t)centre_phase;
    return;
  }

  // analytic distances to the surfaces: near primitives and the nearest surface (normal)
  double x[3];
  for (int d = 0; d < dim; ++d) x[d] = ((double)a[d] + 0.5) / (double)n;
  const double reach = cell.radius_px / (double)n + 1e-9;
  int near[kMaxNear], nnear = 0;
  bool overflow = false;
  double best = 1e300, nrm[3] = {0, 0, 0};
  bool nrm_ok = false;
  int far_first = -1;  // first far primitive that contains the centre (hence the whole ball)
  for (int p = 0; p < cell.nprim; ++p) {
    const FPrim pr = prims[p];
    double dist, vec[3] = {0, 0, 0}, len = 1.0;
    if (pr.kind == HOM_PRIM_SLAB) {
      double d = x[pr.axis] - pr.c[pr.axis];
      d -= rint(d);
      dist = fabs(fabs(d) - 0.5 * pr.radius);
      vec[pr.axis] = 1.0;
    } else {
      double s2 = 0.0;
      for (int d = 0; d < dim; ++d) {
        double t = x[d] - pr.c[d];
        t -= rint(t);
        vec[d] = t;
        s2 += t * t;
      }
      len = sqrt(s2);
      dist = fabs(len - pr.radius);
    }
    if (dist <= reach) {
      if (nnear < kMaxNear) near[nnear++] = p; else overflow = true;
    } else if (far_first < 0 && p >= centre_first && centre_first >= 0 &&
               (p == centre_first || inside_exact(pr, sc, dim, P2, half))) {
      far_first = p;  // contains the centre and no surface crosses the ball: contains every sample
    }
    if (dist < best) {
      best = dist;
      if (pr.kind == HOM_PRIM_SLAB) {
        for (int d = 0; d < 3; ++d) nrm[d] = vec[d];
        nrm_ok = true;
      } else if (len > 1e-12) {
        for (int d = 0; d < 3; ++d) nrm[d] = vec[d] / len;
        nrm_ok = true;
      } else {
        nrm_ok = false;
      }
    }
  }
  if (overflow) { atomicExch(A.err_flag, 2); return; }
  if (nnear == 0) {
    *label = (uint32_t)centre_phase;
    return;
  }

  // count the fine-grid samples of the ball per phase
  const double two_s_r = (2.0 * (double)S) * cell.radius_px;
  const double R2 = two_s_r * two_s_r;
  const int tlo = (int)floor((S - 1 - two_s_r) * 0.5) - 1;
  const int thi = (int)ceil((S - 1 + two_s_r) * 0.5) + 1;
  int ph_id[kMaxPhases], ph_cnt[kMaxPhases], nph = 0;
  long long M = 0;
  const int tz0 = dim == 3 ? tlo : 0, tz1 = dim == 3 ? thi : 0;
  for (int tz = tz0; tz <= tz1; ++tz) {
    const long long Dz = dim == 3 ? (long long)(2 * tz + 1 - S) : 0;
    for (int ty = tlo; ty <= thi; ++ty) {
      const long long Dy = 2 * ty + 1 - S;
      for (int tx = tlo; tx <= thi; ++tx) {
        const long long Dx = 2 * tx + 1 - S;
        const long long q = Dx * Dx + Dy * Dy + Dz * Dz;
        if ((double)q > R2) continue;
        ++M;
        double su[3];
        su[0] = (double)(2 * ((long long)a[0] * S + tx) + 1);
        su[1] = (double)(2 * ((long long)a[1] * S + ty) + 1);
        su[2] = dim == 3 ? (double)(2 * ((long long)a[2] * S + tz) + 1) : 0.0;
        int first = far_first >= 0 ? far_first : 0x7fffffff;
        for (int k = 0; k < nnear; ++k) {
          const int p = near[k];
          if (p >= first) break;  // near[] is sorted by index
          if (inside_exact(prims[p], su, dim, P2, half)) { first = p; break; }
        }
        const int ph = first == 0x7fffffff ? cell.matrix_phase : prims[first].phase;
        int k = 0;
        while (k < nph && ph_id[k] != ph) ++k;
        if (k == nph) {
          if (nph == kMaxPhases) { atomicExch(A.err_flag, 2); return; }
          ph_id[nph] = ph;
          ph_cnt[nph] = 0;
          ++nph;
        }
        ++ph_cnt[k];
      }
    }
  }
  if (nph == 1) {
    *label = (uint32_t)ph_id[0];
    return;
  }
  // sort the present phases by index (deterministic "a < b" order)
  for (int i = 0; i < nph; ++i)
    for (int j = i + 1; j < nph; ++j)
      if (ph_id[j] < ph_id[i]) {
        int t = ph_id[i]; ph_id[i] = ph_id[j]; ph_id[j] = t;
        t = ph_cnt[i]; ph_cnt[i] = ph_cnt[j]; ph_cnt[j] = t;
      }
  const int nc = nc_of(dim), ns = ns_of(dim);
  double Cs[kMaxPhases][36];
  double fs[kMaxPhases];
  for (int k = 0; k < nph; ++k) {
    iso_full_t<double>(A.phase_lame[2 * ph_id[k]], A.phase_lame[2 * ph_id[k] + 1], dim, Cs[k]);
    fs[k] = (double)ph_cnt[k] / (double)M;
  }
  double Ct[36];
  const int rule = apply_rule_t<double>(cell.rule, nph, Cs, fs, nrm_ok, nrm, dim, Ct);
  if (rule < 0) { atomicExch(A.err_flag, 1); return; }
  const unsigned long long m = atomicAdd(A.mixed_counter, 1ull);
  if ((long long)m >= A.mat.mixed_capacity) {
    *label = HOM_MIXED_BIT;  // placeholder: the caller must grow the table and rebuild
    return;
  }
  *label = HOM_MIXED_BIT | (uint32_t)m;
  for (int I = 0; I < nc; ++I)
    for (int J = I; J < nc; ++J) {
      const double val = 0.5 * (Ct[I * nc + J] + Ct[J * nc + I]);
      A.mat.mixed_c64[m * ns + packed_index(nc, I, J)] = val;
      A.mat.mixed_c32[m * ns + packed_index(nc, I, J)] = (float)val;
    }
  A.mat.mixed_phases[2 * m] = ph_id[0];
  A.mat.mixed_phases[2 * m + 1] = ph_id[nph - 1];
  A.mat.mixed_frac[m] = fs[nph - 1];
  for (int d = 0; d < 3; ++d)
    A.mat.mixed_normal[3 * m + d] = (cell.rule == HOM_RULE_TWO_LAYER && rule == HOM_RULE_TWO_LAYER) ? nrm[d] : 0.0;
  A.mat.mixed_voxel[m] = cell.vox_off + v;
}

}  // namespace
}  // namespace hom

using namespace hom;

extern "C" int hom_filter_build(const hom_cell* cells, int32_t ncells, const hom_phase* phases, int32_t nphase,
                                hom_material* mat, void* stream) {
  if (!cells || ncells <= 0 || !phases || nphase <= 0 || !mat)
    return set_error(HOM_ERR_INVALID_ARG, "hom_filter_build: null or empty argument");
  if (mat->nphase != nphase || !mat->label || !mat->phase_c64 || !mat->phase_c32)
    return set_error(HOM_ERR_INVALID_ARG, "hom_filter_build: material buffers missing or nphase mismatch");
  if (mat->mixed_capacity > 0 && (!mat->mixed_c64 || !mat->mixed_c32 || !mat->mixed_phases || !mat->mixed_frac ||
                                  !mat->mixed_normal || !mat->mixed_voxel))
    return set_error(HOM_ERR_INVALID_ARG, "hom_filter_build: mixed-table buffers missing");
  cudaGetLastError();  // do not report an error left behind by an unrelated earlier call
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int dim = cells[0].dim;
  std::vector<FCell> fc(ncells);
  std::vector<FPrim> fp;
  long long vox = 0, blocks = 0;
  for (int c = 0; c < ncells; ++c) {
    const hom_cell& k = cells[c];
    if (k.dim != dim || (dim != 2 && dim != 3))
      return set_error(HOM_ERR_INVALID_ARG, "cell %d: every cell of a call must share dim 2 or 3", c);
    if (!grid_supported(k.n)) return set_error(HOM_ERR_UNSUPPORTED_SIZE, "cell %d: unsupported grid %d", c, k.n);
    if (k.rule < HOM_RULE_NONE || k.rule > HOM_RULE_TWO_LAYER)
      return set_error(HOM_ERR_INVALID_ARG, "cell %d: unknown rule %d", c, k.rule);
    if (k.subgrid < 1 || k.subgrid > 64) return set_error(HOM_ERR_INVALID_ARG, "cell %d: subgrid out of range", c);
    if (!(k.radius_px > 0.0) || k.radius_px > 0.5 * (k.n - 1))
      return set_error(HOM_ERR_INVALID_ARG, "cell %d: filter radius out of range", c);
    if (k.matrix_phase < 0 || k.matrix_phase >= nphase)
      return set_error(HOM_ERR_INVALID_ARG, "cell %d: matrix phase out of range", c);
    if (k.nprim < 0 || (k.nprim > 0 && !k.prims)) return set_error(HOM_ERR_INVALID_ARG, "cell %d: primitives missing", c);
    const double reach = k.rule == HOM_RULE_NONE ? 0.0 : k.radius_px / k.n;
    for (int p = 0; p < k.nprim; ++p) {
      const hom_primitive& q = k.prims[p];
      if (q.phase < 0 || q.phase >= nphase) return set_error(HOM_ERR_INVALID_ARG, "cell %d prim %d: bad phase", c, p);
      if (q.kind == HOM_PRIM_SLAB) {
        if (q.axis < 0 || q.axis >= dim || !(q.radius > 0.0) || !(q.radius < 1.0))
          return set_error(HOM_ERR_INVALID_ARG, "cell %d prim %d: bad slab", c, p);
      } else if ((q.kind == HOM_PRIM_DISK && dim == 2) || (q.kind == HOM_PRIM_SPHERE && dim == 3)) {
        if (!(q.radius > 0.0) || !(q.radius + reach < 0.5))
          return set_error(HOM_ERR_INVALID_ARG, "cell %d prim %d: radius + filter radius must stay below 1/2", c, p);
      } else {
        return set_error(HOM_ERR_INVALID_ARG, "cell %d prim %d: kind %d does not fit dim %d", c, p, q.kind, dim);
      }
      FPrim f{};
      f.kind = q.kind; f.phase = q.phase; f.axis = q.axis;
      for (int d = 0; d < 3; ++d) f.c[d] = q.centre[d];
      f.radius = q.radius;
      fp.push_back(f);
    }
    FCell& f = fc[c];
    f.dim = dim; f.n = k.n; f.matrix_phase = k.matrix_phase; f.rule = k.rule; f.S = k.subgrid;
    f.nprim = k.nprim; f.prim0 = (int)fp.size() - k.nprim; f.radius_px = k.radius_px;
    f.vox_off = vox; f.block0 = blocks;
    const long long nv = (long long)k.n * k.n * (dim == 3 ? k.n : 1);
    vox += nv;
    blocks += (nv + kThreads - 1) / kThreads;
  }
  // phase tables
  const int nc = nc_of(dim), ns = ns_of(dim);
  std::vector<double> lame(2 * (size_t)nphase), pc64((size_t)nphase * ns);
  std::vector<float> pc32((size_t)nphase * ns);
  for (int p = 0; p < nphase; ++p) {
    lame[2 * p] = phases[p].lambda;
    lame[2 * p + 1] = phases[p].mu;
    if (!(phases[p].mu > 0.0) || !(phases[p].lambda + 2.0 * phases[p].mu / dim > 0.0))
      return set_error(HOM_ERR_INVALID_ARG, "phase %d is not positive definite", p);
    for (int I = 0; I < nc; ++I)
      for (int J = I; J < nc; ++J) {
        double v = (I == J) ? 2.0 * phases[p].mu : 0.0;
        if (I < dim && J < dim) v += phases[p].lambda;
        pc64[(size_t)p * ns + packed_index(nc, I, J)] = v;
        pc32[(size_t)p * ns + packed_index(nc, I, J)] = (float)v;
      }
  }
  // scratch: cells, prims, lame, counter, flag
  const size_t b_cells = sizeof(FCell) * ncells, b_prims = sizeof(FPrim) * (fp.size() + 1),
               b_lame = sizeof(double) * lame.size();
  const size_t off_prims = (b_cells + 255) / 256 * 256, off_lame = off_prims + (b_prims + 255) / 256 * 256,
               off_ctr = off_lame + (b_lame + 255) / 256 * 256, total = off_ctr + 256;
  void* ws = nullptr;
  int rc = get_workspace(total, &ws);
  if (rc != HOM_OK) return rc;
  unsigned char* w = static_cast<unsigned char*>(ws);
  std::vector<unsigned char> host(total, 0);
  std::memcpy(host.data(), fc.data(), b_cells);
  if (!fp.empty()) std::memcpy(host.data() + off_prims, fp.data(), sizeof(FPrim) * fp.size());
  std::memcpy(host.data() + off_lame, lame.data(), b_lame);
  HOM_CUDA_TRY(cudaMemcpyAsync(w, host.data(), total, cudaMemcpyHostToDevice, st));
  HOM_CUDA_TRY(cudaMemcpyAsync(mat->phase_c64, pc64.data(), pc64.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  HOM_CUDA_TRY(cudaMemcpyAsync(mat->phase_c32, pc32.data(), pc32.size() * sizeof(float), cudaMemcpyHostToDevice, st));
  FilterArgs args;
  args.cells = reinterpret_cast<const FCell*>(w);
  args.ncells = ncells;
  args.prims = reinterpret_cast<const FPrim*>(w + off_prims);
  args.phase_lame = reinterpret_cast<const double*>(w + off_lame);
  args.nphase = nphase;
  args.mat = *mat;
  args.mixed_counter = reinterpret_cast<unsigned long long*>(w + off_ctr);
  args.err_flag = reinterpret_cast<int*>(w + off_ctr + 8);
  if (blocks > 0x7fffffffLL) return set_error(HOM_ERR_UNSUPPORTED_SIZE, "batch too large");
  k_filter<<<(unsigned)blocks, kThreads, 0, st>>>(args);
  HOM_CUDA_TRY(cudaGetLastError());
  struct { unsigned long long cnt; int flag; int pad; } res{};
  HOM_CUDA_TRY(cudaMemcpyAsync(&res, w + off_ctr, 16, cudaMemcpyDeviceToHost, st));
  HOM_CUDA_TRY(cudaStreamSynchronize(st));
  mat->dim = dim;
  mat->mixed_count = (int64_t)res.cnt;
  if (res.flag == 1) return set_error(HOM_ERR_INVALID_ARG, "2-layer rule met a filter ball holding more than two phases");
  if (res.flag == 2) return set_error(HOM_ERR_INVALID_ARG, "a filter ball meets too many primitives or phases");
  if ((long long)res.cnt > mat->mixed_capacity)
    return set_error(HOM_ERR_CAPACITY, "mixed table needs %llu entries, capacity %lld", res.cnt,
                     (long long)mat->mixed_capacity);
  return HOM_OK;
}

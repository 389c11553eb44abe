// Filtered stiffness c~(x_a) = HR(c, w(x_a)) of section 2 (eqs. 3, 4, 5-a, 5-b).
//
// One CTA covers 256 consecutive voxels of one cell, in three phases:
//   1. one thread per voxel classifies it with FP32 distances to the primitive surfaces: the
//      phase of the voxel centre, the primitives whose surface may cross the filter ball (near),
//      and the first primitive that contains the whole ball.  A voxel with no near primitive is
//      labelled with its centre phase;
//   2. one warp per remaining voxel counts the fine-grid samples of the ball per phase, the
//      lanes splitting the samples;
//   3. one thread per voxel whose samples hold two or more phases computes the 2-layer normal,
//      applies the rule in FP64 and writes a mixed-table entry.
// FP64 arithmetic runs at a small fraction of the FP32 rate on this GPU, so FP64 is kept for
// decisions the FP32 arithmetic cannot settle and for the rule itself.
//
// Exactness.  Sample coordinates are integers in units of h/(2S) (sample 2j+1, voxel centre
// (2a+1)S), and the ball test compares the exact integer sum D^2 with (2 S r)^2.  The membership
// of a sample in a primitive is defined by a fixed sequence of IEEE FP64 operations written with
// explicit round-to-nearest intrinsics (inside_exact).  The FP32 tests below decide only when an
// error bound shows that the FP64 sequence reaches the same answer, and call inside_exact
// otherwise.  The counts therefore equal those of any implementation of that FP64 sequence.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "hom_internal.h"
#include "hom_rules.cuh"

namespace hom {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxNear = 8;     // primitives whose surface can cross one ball
constexpr int kMaxPhases = 4;   // distinct phases inside one ball
// Bound (cell units) used with FP32 surface distances.  The FP32 distance of a voxel centre to a
// surface differs from the exact one by less than 1e-6: the centre (a + 1/2) * (1/n), the primitive
// data and each operation are rounded to FP32 (relative 2^-24 each) on values below 1.
constexpr float kDistMargin = 4e-6f;

__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }

// Wrapped offset su - c * (2 S n) along one axis, in [-S n, S n].  Every operation is exact: cu is
// a double below 2^19 (a multiple of 2^-34) and su an integer, so su - cu and the wrap by 2 S n
// need at most 53 significant bits.
__device__ __forceinline__ double wrapped_offset(double su, double c, double P2, double half) {
  double du = dsub(su, dmul(c, P2));
  if (du > half) du = dsub(du, P2);
  if (du < -half) du = dadd(du, P2);
  return du;
}

// Exact membership of a sample (u-unit coordinates su[0..dim)) in primitive p:
//   du = wrapped offset per axis (above);
//   disk/sphere: ((du_x^2 + du_y^2) + du_z^2) <= (R * 2 S n)^2;  slab: |du_axis| <= T * (S n)
__device__ bool inside_exact(const FPrim& p, const double* su, int dim, double P2, double half) {
  if (p.kind == HOM_PRIM_SLAB) {
    const double du = wrapped_offset(su[p.axis], p.c[p.axis], P2, half);
    return fabs(du) <= dmul(p.radius, half);
  }
  const double Ru = dmul(p.radius, P2);
  const double Ru2 = dmul(Ru, Ru);
  double w = wrapped_offset(su[0], p.c[0], P2, half);
  double q = dmul(w, w);
  for (int ax = 1; ax < dim; ++ax) {
    w = wrapped_offset(su[ax], p.c[ax], P2, half);
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

// A voxel whose ball may meet a surface (phase 1 -> phase 2).
struct NearRec {
  int a[3];                  // voxel coordinates
  int v;                     // flat voxel index within the cell
  int nnear;
  int far_first;             // first primitive containing the whole ball, or -1
  short near[kMaxNear];      // ascending primitive indices
};
// Rule inputs of a mixed voxel, stashed by k_filter in the (not yet written) FP64 stiffness slot
// of its mixed-table entry and read back by k_filter_rule (11 ints: fits the 6 doubles of 2D).
struct RuleStash {
  int cell, nph, nrm_ok;
  int ph[kMaxPhases], cnt[kMaxPhases];
};
static_assert(sizeof(RuleStash) <= 6 * sizeof(double), "stash must fit a 2D entry");

// Per-warp FP32 data of one near primitive for the sample tests of the current voxel.
struct NearPrim {
  float d0[3];               // wrapped offset of the voxel centre, rounded to FP32
  float thr;                 // (R * 2 S n)^2 (disk, sphere) or T * S n (slab), rounded to FP32
  float margin;              // FP32 decisions need |value - thr| > margin
  int axis;                  // slab axis, or -1 for a disk/sphere
};

__global__ void __launch_bounds__(kThreads) k_filter(FilterArgs A) {
  __shared__ NearRec s_near[kThreads];
  __shared__ NearPrim s_np[kWarps][kMaxNear];
  __shared__ int s_nnear;
  __shared__ int s_base[3];
  // locate the cell of this block (cells are few: linear search)
  int ci = 0;
  for (int c = 1; c < A.ncells; ++c)
    if ((long long)blockIdx.x >= A.cells[c].block0) ci = c;
  const FCell& cell = A.cells[ci];
  const int n = cell.n, dim = cell.dim, S = cell.S, nprim = cell.nprim;
  const long long nv = (long long)n * n * (dim == 3 ? n : 1);
  const long long v0 = ((long long)blockIdx.x - cell.block0) * kThreads;
  if (threadIdx.x == 0) {
    s_nnear = 0;
    s_base[0] = (int)(v0 % n);
    s_base[1] = (int)((v0 / n) % n);
    s_base[2] = dim == 3 ? (int)(v0 / ((long long)n * n)) : 0;
  }
  __syncthreads();
  const FPrim* prims = A.prims + cell.prim0;
  const double P2 = 2.0 * (double)S * (double)n;
  const double half = (double)S * (double)n;

  // ---------------------------------------------------------------- 1. classification
  const long long v = v0 + threadIdx.x;
  if (v < nv) {
    int a[3];
    {
      const int t0 = s_base[0] + (int)threadIdx.x;
      const int q0 = fdiv(t0, cell.dn);
      a[0] = t0 - q0 * n;
      const int t1 = s_base[1] + q0;
      const int q1 = fdiv(t1, cell.dn);
      a[1] = t1 - q1 * n;
      a[2] = s_base[2] + q1;
    }
    float xf[3];
    for (int d = 0; d < dim; ++d) xf[d] = ((float)a[d] + 0.5f) * cell.inv_n;
    const bool filtered = cell.rule != HOM_RULE_NONE;
    const float near_lim = cell.reach32 + kDistMargin;
    int centre_first = -1, far_first = -1, nnear = 0;
    short near[kMaxNear];
    bool overflow = false;
    for (int p = 0; p < nprim; ++p) {
      const FPrim& pr = prims[p];
      float dist;
      bool in32;
      if (pr.kind == HOM_PRIM_SLAB) {
        float d = xf[pr.axis] - pr.c32[pr.axis];
        d -= rintf(d);
        const float ad = fabsf(d), th = 0.5f * pr.r32;
        dist = fabsf(ad - th);
        in32 = ad < th;
      } else {
        float s2 = 0.f;
        for (int d = 0; d < dim; ++d) {
          float t = xf[d] - pr.c32[d];
          t -= rintf(t);
          s2 = fmaf(t, t, s2);
        }
        const float len = sqrtf(s2);
        dist = fabsf(len - pr.r32);
        in32 = len < pr.r32;
      }
      // phase of the centre: FP32 decides when the centre is clearly off the surface
      if (centre_first < 0) {
        bool in = in32;
        if (dist <= kDistMargin) {
          double sc[3];
          for (int d = 0; d < dim; ++d) sc[d] = (double)(2 * a[d] + 1) * (double)S;
          in = inside_exact(pr, sc, dim, P2, half);
        }
        if (in) centre_first = p;
      }
      if (!filtered) {
        if (centre_first >= 0) break;
        continue;
      }
      // near primitives after far_first own no sample but may hold the nearest surface (normal)
      if (dist <= near_lim) {
        if (nnear < kMaxNear) near[nnear++] = (short)p; else overflow = true;
      } else if (in32 && far_first < 0) {
        far_first = p;  // contains the centre and no surface crosses the ball: contains every sample
      }
    }
    const int centre_phase = centre_first >= 0 ? prims[centre_first].phase : cell.matrix_phase;
    uint32_t* label = A.mat.label + cell.vox_off + v;
    if (overflow) {
      atomicExch(A.err_flag, 2);
      *label = (uint32_t)centre_phase;
    } else if (!filtered || nnear == 0) {
      *label = (uint32_t)centre_phase;
    } else {
      const int r = atomicAdd(&s_nnear, 1);
      NearRec& rec = s_near[r];
      for (int d = 0; d < 3; ++d) rec.a[d] = a[d];
      rec.v = (int)(v - v0);
      rec.nnear = nnear;
      rec.far_first = far_first;
      for (int k = 0; k < kMaxNear; ++k) rec.near[k] = k < nnear ? near[k] : (short)0;
    }
  }
  __syncthreads();

  // ---------------------------------------------------------------- 2. sample counts, one warp per voxel
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nt = cell.thi - cell.tlo + 1;
  const int total = dim == 3 ? nt * nt * nt : nt * nt;
  // largest |offset| of a ball sample from the voxel centre, in h/(2S) units
  const int offmax = max(abs(2 * cell.tlo + 1 - S), abs(2 * cell.thi + 1 - S));
  for (int r = warp; r < s_nnear; r += kWarps) {
    const NearRec& rec = s_near[r];
    const int nnear = rec.nnear;
    if (lane < nnear) {
      // FP32 data of near primitive `lane`.  Bounds (u = h/(2S) units, B = S n + offmax): a sample
      // offset du32 = fl(fl(d0) + off) is within e = 2^-23 B of the exact wrapped offset; the FP32
      // squared distance is then within dim B^2 2^-21 of the exact sum, and the FP64 sum within a
      // relative 2^-50 of it.  The margins below are twice these bounds.
      const FPrim& pr = prims[rec.near[lane]];
      NearPrim np;
      for (int d = 0; d < 3; ++d) {
        np.d0[d] = d < dim ? (float)wrapped_offset((double)(2 * rec.a[d] + 1) * (double)S, pr.c[d], P2, half)
                           : 0.f;
      }
      const float B = (float)half + (float)offmax;
      if (pr.kind == HOM_PRIM_SLAB) {
        np.axis = pr.axis;
        np.thr = (float)dmul(pr.radius, half);
        np.margin = ldexpf(B + np.thr, -21);
      } else {
        np.axis = -1;
        const double Ru = dmul(pr.radius, P2);
        np.thr = (float)dmul(Ru, Ru);
        np.margin = (float)dim * B * B * ldexpf(1.f, -20) + ldexpf(np.thr, -22);
      }
      s_np[warp][lane] = np;
    }
    __syncwarp();
    const int far_first = rec.far_first;
    const float wrap_guard = (float)half - 2.f;
    int cnt[kMaxNear + 1];
#pragma unroll
    for (int k = 0; k <= kMaxNear; ++k) cnt[k] = 0;
    for (int i = lane; i < total; i += 32) {
      int t[3];
      const int q = fdiv(i, cell.dnt);
      t[0] = i - q * nt;
      if (dim == 3) {
        const int q2 = fdiv(q, cell.dnt);
        t[1] = q - q2 * nt;
        t[2] = q2;
      } else {
        t[1] = q;
        t[2] = 0;
      }
      int D[3], q2sum = 0;
      for (int d = 0; d < 3; ++d) {
        D[d] = d < dim ? 2 * (t[d] + cell.tlo) + 1 - S : 0;
        q2sum += D[d] * D[d];
      }
      if (q2sum > cell.R2i) continue;
      int slot = 0;  // 0: no near primitive contains the sample; k + 1: near primitive k
      for (int k = 0; k < nnear; ++k) {
        const int p = rec.near[k];
        if (far_first >= 0 && p > far_first) break;
        const NearPrim& np = s_np[warp][k];
        int verdict;  // 1 inside, 0 outside, -1 undecided in FP32
        if (np.axis >= 0) {
          const float u = np.d0[np.axis] + (float)D[np.axis];
          const float au = fabsf(u);
          if (au > wrap_guard) verdict = -1;
          else verdict = au <= np.thr - np.margin ? 1 : (au > np.thr + np.margin ? 0 : -1);
        } else {
          const float u0 = np.d0[0] + (float)D[0];
          const float u1 = np.d0[1] + (float)D[1];
          const float u2 = np.d0[2] + (float)D[2];
          if (fmaxf(fabsf(u0), fmaxf(fabsf(u1), fabsf(u2))) > wrap_guard) {
            verdict = -1;
          } else {
            const float q32 = fmaf(u2, u2, fmaf(u1, u1, u0 * u0));
            verdict = q32 <= np.thr - np.margin ? 1 : (q32 > np.thr + np.margin ? 0 : -1);
          }
        }
        if (verdict < 0) {
          double su[3];
          for (int d = 0; d < dim; ++d) su[d] = (double)(2 * ((rec.a[d] * S) + t[d] + cell.tlo) + 1);
          verdict = inside_exact(prims[p], su, dim, P2, half) ? 1 : 0;
        }
        if (verdict) {
          slot = k + 1;
          break;
        }
      }
#pragma unroll
      for (int k = 0; k <= kMaxNear; ++k) cnt[k] += slot == k ? 1 : 0;
    }
#pragma unroll
    for (int k = 0; k <= kMaxNear; ++k)
      for (int o = 16; o > 0; o >>= 1) cnt[k] += __shfl_xor_sync(0xffffffffu, cnt[k], o);
    if (lane == 0) {
      int ph_id[kMaxPhases], ph_cnt[kMaxPhases], nph = 0;
      bool too_many = false;
      for (int k = 0; k <= nnear; ++k) {
        if (cnt[k] == 0) continue;
        const int ph = k == 0 ? (far_first >= 0 ? prims[far_first].phase : cell.matrix_phase)
                              : prims[rec.near[k - 1]].phase;
        int j = 0;
        while (j < nph && ph_id[j] != ph) ++j;
        if (j == nph) {
          if (nph == kMaxPhases) { too_many = true; break; }
          ph_id[nph] = ph;
          ph_cnt[nph] = 0;
          ++nph;
        }
        ph_cnt[j] += cnt[k];
      }
      uint32_t* label = A.mat.label + cell.vox_off + v0 + rec.v;
      if (too_many) {
        atomicExch(A.err_flag, 2);
        *label = (uint32_t)ph_id[0];
      } else if (nph == 1) {
        *label = (uint32_t)ph_id[0];
      } else if (cell.rule == HOM_RULE_TWO_LAYER && nph > 2) {
        atomicExch(A.err_flag, 1);
        *label = (uint32_t)ph_id[0];
      } else {
        // 2-layer normal: unit vector from the centre of the primitive whose surface is nearest
        // to x_a (first one on ties), or the slab normal.  That primitive is a near one.
        double nrm[3] = {0, 0, 0};
        bool nrm_ok = false;
        if (cell.rule == HOM_RULE_TWO_LAYER) {
          double x[3];
          for (int d = 0; d < dim; ++d) x[d] = ((double)rec.a[d] + 0.5) / (double)n;
          double best = 1e300;
          for (int k = 0; k < nnear; ++k) {
            const FPrim& pr = prims[rec.near[k]];
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
        }
        const unsigned long long m = atomicAdd(A.mixed_counter, 1ull);
        if ((long long)m >= A.mat.mixed_capacity) {
          *label = HOM_MIXED_BIT;  // placeholder: the caller must grow the table and rebuild
        } else {
          *label = HOM_MIXED_BIT | (uint32_t)m;
          RuleStash st;
          st.cell = ci;
          st.nph = nph;
          st.nrm_ok = nrm_ok ? 1 : 0;
          for (int j = 0; j < kMaxPhases; ++j) {
            st.ph[j] = j < nph ? ph_id[j] : 0;
            st.cnt[j] = j < nph ? ph_cnt[j] : 0;
          }
          *reinterpret_cast<RuleStash*>(A.mat.mixed_c64 + m * ns_of(dim)) = st;
          for (int d = 0; d < 3; ++d) A.mat.mixed_normal[3 * m + d] = nrm[d];
          A.mat.mixed_voxel[m] = cell.vox_off + v0 + rec.v;
        }
      }
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------- rule, one thread per mixed entry
__global__ void __launch_bounds__(kThreads) k_filter_rule(FilterArgs A) {
  const long long m = (long long)blockIdx.x * kThreads + threadIdx.x;
  const unsigned long long cnt_all = *A.mixed_counter;
  if (m >= A.mat.mixed_capacity || (unsigned long long)m >= cnt_all) return;
  const int dim = A.mat.dim;
  const int nc = nc_of(dim), ns = ns_of(dim);
  const RuleStash st = *reinterpret_cast<const RuleStash*>(A.mat.mixed_c64 + m * ns);
  const FCell& cell = A.cells[st.cell];
  int ph_id[kMaxPhases], ph_cnt[kMaxPhases];
  const int nph = st.nph;
  for (int j = 0; j < kMaxPhases; ++j) {
    ph_id[j] = st.ph[j];
    ph_cnt[j] = st.cnt[j];
  }
  // sort the present phases by index (deterministic "a < b" order)
  for (int i = 0; i < nph; ++i)
    for (int j = i + 1; j < nph; ++j)
      if (ph_id[j] < ph_id[i]) {
        int t = ph_id[i]; ph_id[i] = ph_id[j]; ph_id[j] = t;
        t = ph_cnt[i]; ph_cnt[i] = ph_cnt[j]; ph_cnt[j] = t;
      }
  double nrm[3];
  for (int d = 0; d < 3; ++d) nrm[d] = A.mat.mixed_normal[3 * m + d];
  double Cs[kMaxPhases][36];
  double fs[kMaxPhases];
  for (int k = 0; k < nph; ++k) {
    iso_full_t<double>(A.phase_lame[2 * ph_id[k]], A.phase_lame[2 * ph_id[k] + 1], dim, Cs[k]);
    fs[k] = (double)ph_cnt[k] / (double)cell.M;
  }
  double Ct[36];
  const int rule = apply_rule_t<double>(cell.rule, nph, Cs, fs, st.nrm_ok != 0, nrm, dim, Ct);
  for (int I = 0; I < nc; ++I)
    for (int J = I; J < nc; ++J) {
      const double val = 0.5 * (Ct[I * nc + J] + Ct[J * nc + I]);
      A.mat.mixed_c64[m * ns + packed_index(nc, I, J)] = val;
      A.mat.mixed_c32[m * ns + packed_index(nc, I, J)] = (float)val;
    }
  A.mat.mixed_phases[2 * m] = ph_id[0];
  A.mat.mixed_phases[2 * m + 1] = ph_id[nph - 1];
  A.mat.mixed_frac[m] = fs[nph - 1];
  if (!(cell.rule == HOM_RULE_TWO_LAYER && rule == HOM_RULE_TWO_LAYER))
    for (int d = 0; d < 3; ++d) A.mat.mixed_normal[3 * m + d] = 0.0;
}

}  // namespace
}  // namespace hom

using namespace hom;

extern "C" int hom_filter_build(const hom_cell* cells, int32_t ncells, const hom_phase* phases, int32_t nphase,
                                hom_material* mat, void* stream) {
  ::hom::NvtxRange nvtx_range_("hom_filter_build");
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
      for (int d = 0; d < 3; ++d) f.c32[d] = (float)q.centre[d];
      f.r32 = (float)q.radius;
      fp.push_back(f);
    }
    FCell& f = fc[c];
    f.dim = dim; f.n = k.n; f.matrix_phase = k.matrix_phase; f.rule = k.rule; f.S = k.subgrid;
    f.nprim = k.nprim; f.prim0 = (int)fp.size() - k.nprim; f.radius_px = k.radius_px;
    f.vox_off = vox; f.block0 = blocks;
    f.inv_n = (float)(1.0 / k.n);
    f.reach32 = (float)(k.radius_px / k.n);
    f.dn = make_fastdiv(k.n);
    // fine points of a ball: offsets t (j = a S + t) with D = 2t + 1 - S and sum D^2 <= (2 S r)^2
    const double two_s_r = (2.0 * k.subgrid) * k.radius_px;
    const double R2 = two_s_r * two_s_r;
    f.tlo = (int)std::floor((k.subgrid - 1 - two_s_r) * 0.5) - 1;
    f.thi = (int)std::ceil((k.subgrid - 1 + two_s_r) * 0.5) + 1;
    const long long nt = f.thi - f.tlo + 1;
    long long pw = nt;
    for (int d = 0; d < dim; ++d) pw *= nt;
    if (k.rule != HOM_RULE_NONE && pw >= (1LL << 32))
      return set_error(HOM_ERR_UNSUPPORTED_SIZE, "cell %d: filter ball too large for the sampler (subgrid x radius)", c);
    f.R2i = k.rule != HOM_RULE_NONE ? (int)std::floor(R2) : 0;
    f.dnt = make_fastdiv((int)nt);
    f.M = 0;
    if (k.rule != HOM_RULE_NONE) {
      const long long tot = dim == 3 ? nt * nt * nt : nt * nt;
      for (long long i = 0; i < tot; ++i) {
        long long r = i, q = 0;
        for (int d = 0; d < dim; ++d) {
          const long long D = 2 * (r % nt + f.tlo) + 1 - k.subgrid;
          q += D * D;
          r /= nt;
        }
        if ((double)q <= R2) ++f.M;
      }
    }
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
  args.mat.dim = dim;
  k_filter<<<(unsigned)blocks, kThreads, 0, st>>>(args);
  HOM_CUDA_TRY(cudaGetLastError());
  if (mat->mixed_capacity > 0) {
    const long long rblocks = (mat->mixed_capacity + kThreads - 1) / kThreads;
    if (rblocks > 0x7fffffffLL) return set_error(HOM_ERR_UNSUPPORTED_SIZE, "mixed table too large");
    k_filter_rule<<<(unsigned)rblocks, kThreads, 0, st>>>(args);
    HOM_CUDA_TRY(cudaGetLastError());
  }
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

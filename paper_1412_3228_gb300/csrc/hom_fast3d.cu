// Specialised FP32 passes of the 3D fixed-point scheme (section 2, eqs. 1-a, 1-b, 2) for grid
// sizes n with a compile-time radix plan (27, 45, 81, 135, 243).  Same lane-pair scheme as the 2D
// passes (hom_fast2d.cu): shared memory holds float4 (re_A, re_B, im_A, im_B) per (position,
// component), with the six Mandel components side by side; positions are 7 float4 apart in shared
// memory (112 bytes: neighbouring threads' 16-byte accesses fall on distinct bank quads).
//
// One iteration is four passes, as in the generic 3D path:
//   row pass   : 4 real rows (same z, consecutive y) x every active load; lines A = rows 0 + i 1,
//                B = rows 2 + i 3; inverse x-DFT, constitutive update, forward x-DFT (tau);
//   y forward  : one load, one kx pair, one z: forward y-DFT of tau in place (bins left at
//                digit-reversed positions);
//   Green pass : one load, one kx pair, one y position: forward z-DFT, Gamma0 and the residual on J
//                (eq. 2), inverse z-DFT, in place;
//   y inverse  : inverse y-DFT (digit-reversed -> natural) into the next eps buffer.
//
// State in HBM is tiled by kx pairs: [load][kx pair][z][y][component] float4 lane pairs, so a row
// task reads 4 x 96 contiguous bytes per pair and a y task one contiguous tile; the Green pass
// gathers 96-byte pieces with 16-byte asynchronous copies.  The displacement-like state g of the
// Green pass is private: [load][kx pair][y position][z position][3 lane pairs].
#define HOM_FILE_ID 3
#include <algorithm>

#include "hom_fast2d.h"
#include "hom_solve_args.cuh"
#include "hom_fastfft.cuh"
#include "hom_em.cuh"

namespace hom {
namespace {

constexpr int NP = 6;                       // lane pairs per position (3D Mandel components)
constexpr int SP = 7;                       // shared-memory position stride (float4): 28 words keeps
                                            // 8 neighbouring 16-byte accesses on distinct bank quads
constexpr int kSizes3[] = {27, 45, 81, 135, 243};
#ifndef HOM_FAST3D_THREADS
#define HOM_FAST3D_THREADS 128
#endif
constexpr int kT3 = HOM_FAST3D_THREADS;     // threads per CTA: the 3D lines (n <= 243) give few
                                            // butterflies per stage, so smaller CTAs idle less
constexpr int kMinB3 = 768 / kT3;           // resident CTAs per SM the register budget targets
constexpr uint32_t kLabel8Mixed = 255;      // one-byte label of a mixed voxel

__device__ __forceinline__ size_t idx3(const CellDev& c, int n, int l, int p, int z, int y) {
  return (size_t)c.ws_off / 2 + ((((size_t)l * (c.Hp / 2) + p) * n + z) * n + y) * NP;
}

// ------------------------------------------------------------------ row pass
struct RowShared3 {
  int al[kMaxLoads], nal;
  float dc[kMaxLoads][2][kFastRows][NP];  // [load][eps row mean, tau row sum][row][comp]
};

constexpr int kRowSpare3 = 2 * NP * kFastRows;  // float4 entries of the row pass's spare landing area

// EM (Eyre-Milton scheme): as in the 2D row pass, the state is u = sigma + c0 : eps; pure voxels take
// tau = W u with a per-phase isotropic W, mixed groups and the output pass solve eps = (c~ + c0)^-1 u
// first, and the row sums of sigma are (tau + u) / 2.
template <int N, bool OUT, bool SRC, bool EM = false>
__device__ __forceinline__ void row3_body(const SolveArgs& A, int task, const TaskR& t, const CellDev& c,
                                          const FastPlanDev& fp, float4* s, RowShared3& sh) {
  constexpr int H = (N + 1) / 2;
  constexpr int P = (H + 1) / 2;
  constexpr int NL = (N + 15) / 16 * 16;
  const int it = *A.it_dev;
  if (threadIdx.x == 0) {
    int nal = 0;
    for (int l = 0; l < A.L; ++l)
      if ((t.load < 0 || l == t.load) && (OUT || A.active[t.cell * A.L + l])) sh.al[nal++] = l;
    sh.nal = nal;
  }
  __syncthreads();
  const int nal = sh.nal;
  if (nal == 0) return;
  const int z = t.row0 / N, y0 = t.row0 - z * N, nr = t.nrows;
  CellConst<float> cc;
  cell_const(c, cc);
  const float lam0 = OUT ? 0.f : cc.lam0, mu2_0 = OUT ? 0.f : cc.mu2;
  float4* taub = static_cast<float4*>(A.tau);
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  uint8_t* slab = reinterpret_cast<uint8_t*>(s + N * SP);
  {
    const uint4* src = reinterpret_cast<const uint4*>(A.label8 + c.lp_off + (size_t)t.row0 * NL);
    for (int i = threadIdx.x; i < nr * NL / 16; i += kT3) cp16(slab + 16 * i, src + i);
  }
  float2* tws = reinterpret_cast<float2*>(s + N * SP + kFastRows * NL / 16);
  for (int i = threadIdx.x; i < (N + 1) / 2; i += kT3) cp16(tws + 2 * i, fp.tw2 + 2 * i);
  float4* spare = s + N * SP + kFastRows * NL / 16 + (N + 1) / 2;
  float2* sph = reinterpret_cast<float2*>(spare + kRowSpare3);
  float2* sinv = sph + c.nph;  // EM: per local phase, (c + c0)^-1 as (coefficient of tr(u) I, of u)
  cp_commit();
  for (int i = threadIdx.x; i < c.nph; i += kT3) {
    const float* pc = A.phase_c32 + (size_t)__ldg(A.cell_phases + c.ph_off + i) * 21;
    const float lam = __ldg(pc + 1);
    const float mu2 = __ldg(pc) - lam;
    sph[i] = make_float2(lam - lam0, mu2 - mu2_0);
    if (EM) {
      // (c + c0)^-1: volumetric eigenvalue 3 (lam + lam0) + (2 mu + 2 mu0), deviatoric 2 mu + 2 mu0
      const double l = (double)lam, m2 = (double)mu2, l0 = c.lam0, m20 = 2.0 * c.mu0;
      const double ms2 = m2 + m20, ks = 3.0 * (l + l0) + ms2;
      sinv[i] = make_float2((float)((1.0 / ks - 1.0 / ms2) / 3.0), (float)(1.0 / ms2));
      if (!OUT) {  // W = (c - c0)(c + c0)^-1
        const double aK = (m2 - m20) / ms2, aJ = (3.0 * (l - l0) + (m2 - m20)) / ks;
        sph[i] = make_float2((float)((aJ - aK) / 3.0), (float)aK);
      }
    }
  }

  for (int la = 0; la < nal; ++la) {
    const int l = sh.al[la];
    const float4* ein = static_cast<const float4*>(A.eps[OUT ? (A.iters[t.cell * A.L + l] & 1) : (it & 1)]);
    // 1. four half-spectrum rows -> two Hermitian-extended lines per component: the row values of
    // item (p, k) land by asynchronous copies in the slots of the line positions they produce
    // (row_slot_p) and are expanded in place (see the 2D row pass)
    for (int f = threadIdx.x; f < P * NP; f += kT3) {
      const int p = f / NP, k = f - p * NP;
      const float4* src = ein + idx3(c, N, l, p, z, y0) + k;
#pragma unroll
      for (int r = 0; r < kFastRows; ++r)
        cp16z(row_slot_p<N, NP, SP>(s, spare, p, k, r), src + (size_t)(r < nr ? r : 0) * NP, r < nr ? 16u : 0u);
    }
    cp_commit();
    if (la + 1 < nal) {  // the next active load's rows -> L2
      const int ln = sh.al[la + 1];
      const float4* nx = static_cast<const float4*>(A.eps[OUT ? (A.iters[t.cell * A.L + ln] & 1) : (it & 1)]);
      for (int p = threadIdx.x; p < P; p += kT3)
        prefetch_l2(nx + idx3(c, N, ln, p, z, y0), (unsigned)(nr * NP * sizeof(float4)));
    }
    cp_wait_all();
    __syncthreads();
    for (int f = threadIdx.x; f < P * NP; f += kT3) {
      const int p = f / NP, k = f - p * NP;
      float4 v[kFastRows];
#pragma unroll
      for (int r = 0; r < kFastRows; ++r) v[r] = *row_slot_p<N, NP, SP>(s, spare, p, k, r);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int kx = 2 * p + h;
        if (kx >= H) break;
        const float2 q0 = h ? make_float2(v[0].y, v[0].w) : make_float2(v[0].x, v[0].z);
        const float2 q1 = h ? make_float2(v[1].y, v[1].w) : make_float2(v[1].x, v[1].z);
        const float2 q2 = h ? make_float2(v[2].y, v[2].w) : make_float2(v[2].x, v[2].z);
        const float2 q3 = h ? make_float2(v[3].y, v[3].w) : make_float2(v[3].x, v[3].z);
        s[kx * SP + k] = make_float4(q0.x - q1.y, q2.x - q3.y, q0.y + q1.x, q2.y + q3.x);
        if (kx > 0) {
          s[(N - kx) * SP + k] = make_float4(q0.x + q1.y, q2.x + q3.y, q1.x - q0.y, q3.x - q2.y);
        } else {
          sh.dc[la][0][0][k] = q0.x;
          sh.dc[la][0][1][k] = q1.x;
          sh.dc[la][0][2][k] = q2.x;
          sh.dc[la][0][3][k] = q3.x;
        }
      }
    }
    __syncthreads();
    fft_dif_p<NP, N, false, float2, SP, kT3>(s, tws);  // inverse: eps at digit-reversed positions

    // 2. constitutive update; lanes (x, y, z, w) of a float4 are rows (0, 2, 1, 3)
    for (int pos = threadIdx.x; pos < N; pos += kT3) {
      uint32_t lab[kFastRows];
      bool mixed = false;
#pragma unroll
      for (int r = 0; r < kFastRows; ++r) {
        lab[r] = r < nr ? (uint32_t)slab[r * NL + pos] : 0u;
        mixed |= lab[r] == kLabel8Mixed;
      }
      float4 e[NP], o[NP];
#pragma unroll
      for (int k = 0; k < NP; ++k) e[k] = s[pos * SP + k];
      if (EM && (OUT || mixed)) {
        // e holds u: eps = (c~ + c0)^-1 u per voxel (mixed: the per-call table; pure: closed form)
        const int x = __ldg(fp.iperm + pos);
#pragma unroll
        for (int r = 0; r < kFastRows; ++r) {
          float u[NP], ev[NP];
#pragma unroll
          for (int k = 0; k < NP; ++k) u[k] = r == 0 ? e[k].x : r == 1 ? e[k].z : r == 2 ? e[k].y : e[k].w;
          const uint32_t L = !mixed ? 0u : lab[r] == kLabel8Mixed ? __ldg(A.label + c.vox_off + (size_t)(t.row0 + r) * N + x)
                                                                  : (uint32_t)__ldg(A.cell_phases + c.ph_off + lab[r]);
          if (mixed && (L & HOM_MIXED_BIT)) {
            const float* M = static_cast<const float*>(A.em_minv) + (size_t)(L & ~HOM_MIXED_BIT) * 21;
#pragma unroll
            for (int I = 0; I < NP; ++I) {
              float acc = 0.f;
#pragma unroll
              for (int J = 0; J < NP; ++J) acc = fmaf(__ldg(M + packed_index(NP, I, J)), u[J], acc);
              ev[I] = acc;
            }
          } else {
            float2 d;
            if (lab[r] == kLabel8Mixed) {  // a pure voxel whose phase is not in the cell's list (rare)
              const float* pc = A.phase_c32 + (size_t)L * 21;
              const float l = __ldg(pc + 1), m2 = __ldg(pc) - l;
              const float ms2 = m2 + cc.mu2, ks = 3.f * (l + cc.lam0) + ms2;
              d = make_float2((1.f / ks - 1.f / ms2) / 3.f, 1.f / ms2);
            } else {
              d = sinv[lab[r]];
            }
            const float tr = u[0] + u[1] + u[2];
#pragma unroll
            for (int k = 0; k < NP; ++k) ev[k] = d.y * u[k] + (k < 3 ? d.x * tr : 0.f);
          }
#pragma unroll
          for (int k = 0; k < NP; ++k) {
            if (r == 0) e[k].x = ev[k];
            else if (r == 1) e[k].z = ev[k];
            else if (r == 2) e[k].y = ev[k];
            else e[k].w = ev[k];
          }
        }
      }
      if (!mixed) {
        float2 dl_lo, dl_hi, dm_lo, dm_hi;
        {
          const float2 d0 = sph[lab[0]], d1 = sph[lab[1]], d2 = sph[lab[2]], d3 = sph[lab[3]];
          dl_lo = make_float2(d0.x, d2.x);
          dl_hi = make_float2(d1.x, d3.x);
          dm_lo = make_float2(d0.y, d2.y);
          dm_hi = make_float2(d1.y, d3.y);
        }
        const float2 tr_lo = add2(add2(make_float2(e[0].x, e[0].y), make_float2(e[1].x, e[1].y)),
                                  make_float2(e[2].x, e[2].y));
        const float2 tr_hi = add2(add2(make_float2(e[0].z, e[0].w), make_float2(e[1].z, e[1].w)),
                                  make_float2(e[2].z, e[2].w));
#pragma unroll
        for (int k = 0; k < NP; ++k) {
          float2 lo = mul2(dm_lo, make_float2(e[k].x, e[k].y));
          float2 hi = mul2(dm_hi, make_float2(e[k].z, e[k].w));
          if (k < 3) {
            lo = fma2(dl_lo, tr_lo, lo);
            hi = fma2(dl_hi, tr_hi, hi);
          }
          o[k] = make_float4(lo.x, lo.y, hi.x, hi.y);
        }
      } else {
        const int x = __ldg(fp.iperm + pos);
        float out[NP][kFastRows];
#pragma unroll
        for (int r = 0; r < kFastRows; ++r) {
          const uint32_t L = lab[r] == kLabel8Mixed ? __ldg(A.label + c.vox_off + (size_t)(t.row0 + r) * N + x)
                                                    : (uint32_t)__ldg(A.cell_phases + c.ph_off + lab[r]);
          const float* src = (L & HOM_MIXED_BIT) ? A.mixed_c32 + (size_t)(L & ~HOM_MIXED_BIT) * 21
                                                 : A.phase_c32 + (size_t)L * 21;
          float ev[NP];
#pragma unroll
          for (int k = 0; k < NP; ++k) ev[k] = r == 0 ? e[k].x : r == 1 ? e[k].z : r == 2 ? e[k].y : e[k].w;
          const float tr0 = ev[0] + ev[1] + ev[2];
#pragma unroll
          for (int I = 0; I < NP; ++I) {
            float sg = 0.f;
#pragma unroll
            for (int J = 0; J < NP; ++J) sg = fmaf(__ldg(src + packed_index(NP, I, J)), ev[J], sg);
            out[I][r] = sg - (mu2_0 * ev[I] + (I < 3 ? lam0 * tr0 : 0.f));
          }
        }
#pragma unroll
        for (int k = 0; k < NP; ++k) o[k] = make_float4(out[k][0], out[k][2], out[k][1], out[k][3]);
      }
      if constexpr (SRC) {
        // adjoint solve: tau = (c~ - c0) : w - c~ : S, the source S (real field, solver output
        // layout) read at the rows' voxels
        const int x = __ldg(fp.iperm + pos);
        const float* Sb = static_cast<const float*>(A.src) + c.fld_off + (size_t)l * NP * c.nv + (size_t)t.row0 * N + x;
#pragma unroll
        for (int r = 0; r < kFastRows; ++r) {
          if (r >= nr) break;
          const uint32_t L = lab[r] == kLabel8Mixed ? __ldg(A.label + c.vox_off + (size_t)(t.row0 + r) * N + x)
                                                    : (uint32_t)__ldg(A.cell_phases + c.ph_off + lab[r]);
          const float* C = (L & HOM_MIXED_BIT) ? A.mixed_c32 + (size_t)(L & ~HOM_MIXED_BIT) * 21 : A.phase_c32 + (size_t)L * 21;
          float sv[NP];
#pragma unroll
          for (int k = 0; k < NP; ++k) sv[k] = __ldg(Sb + (size_t)k * c.nv + (size_t)r * N);
#pragma unroll
          for (int I = 0; I < NP; ++I) {
            float cs = 0.f;
#pragma unroll
            for (int J = 0; J < NP; ++J) cs = fmaf(__ldg(C + packed_index(NP, I, J)), sv[J], cs);
            if (r == 0) o[I].x -= cs;
            else if (r == 1) o[I].z -= cs;
            else if (r == 2) o[I].y -= cs;
            else o[I].w -= cs;
          }
        }
      }
      if (OUT) {
        const int x = __ldg(fp.iperm + pos);
        float* oe = static_cast<float*>(A.out_eps);
        float* os = static_cast<float*>(A.out_sig);
        const size_t base = c.fld_off + (size_t)l * NP * c.nv + (size_t)t.row0 * N + x;
#pragma unroll
        for (int r = 0; r < kFastRows; ++r) {
          if (r >= nr) break;
#pragma unroll
          for (int k = 0; k < NP; ++k) {
            const float ev = r == 0 ? e[k].x : r == 1 ? e[k].z : r == 2 ? e[k].y : e[k].w;
            const float sv = r == 0 ? o[k].x : r == 1 ? o[k].z : r == 2 ? o[k].y : o[k].w;
            const size_t ad = base + (size_t)k * c.nv + (size_t)r * N;
            if (oe) oe[ad] = ev;
            if (os) os[ad] = sv;
          }
        }
      } else {
#pragma unroll
        for (int k = 0; k < NP; ++k) s[pos * SP + k] = o[k];
      }
    }
    __syncthreads();  // the tile is read above and rewritten below (or by the next load's fill)
    if (OUT) continue;
    fft_dit_p<NP, N, true, float2, SP, kT3>(s, tws);  // forward: natural order

    // 3. split the two real rows of each line; store the half spectra of tau pair by pair
    for (int f = threadIdx.x; f < P * NP; f += kT3) {
      const int p = f / NP, k = f - p * NP;
      float4 w[kFastRows];
#pragma unroll
      for (int r = 0; r < kFastRows; ++r) w[r] = z4;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int kx = 2 * p + h;
        if (kx >= H) break;
        const float4 Z = s[kx * SP + k];
        const float4 Zm = s[(kx == 0 ? 0 : N - kx) * SP + k];
        const float2 o0 = make_float2(0.5f * (Z.x + Zm.x), 0.5f * (Z.z - Zm.z));
        const float2 o1 = make_float2(0.5f * (Z.z + Zm.z), 0.5f * (Zm.x - Z.x));
        const float2 o2 = make_float2(0.5f * (Z.y + Zm.y), 0.5f * (Z.w - Zm.w));
        const float2 o3 = make_float2(0.5f * (Z.w + Zm.w), 0.5f * (Zm.y - Z.y));
        if (h == 0) {
          w[0].x = o0.x; w[0].z = o0.y; w[1].x = o1.x; w[1].z = o1.y;
          w[2].x = o2.x; w[2].z = o2.y; w[3].x = o3.x; w[3].z = o3.y;
          if (kx == 0) {
            sh.dc[la][1][0][k] = o0.x;
            sh.dc[la][1][1][k] = o1.x;
            sh.dc[la][1][2][k] = o2.x;
            sh.dc[la][1][3][k] = o3.x;
          }
        } else {
          w[0].y = o0.x; w[0].w = o0.y; w[1].y = o1.x; w[1].w = o1.y;
          w[2].y = o2.x; w[2].w = o2.y; w[3].y = o3.x; w[3].w = o3.y;
        }
      }
      const size_t b = idx3(c, N, l, p, z, y0) + k;
#pragma unroll
      for (int r = 0; r < kFastRows; ++r)
        if (r < nr) taub[b + (size_t)r * NP] = w[r];
    }
    __syncthreads();
  }
  if (OUT) {
    if (threadIdx.x == 0)
      atomicAdd(A.bytes + HOM_K_OUTPUT,
                (unsigned long long)((size_t)nal * nr * NP * (H * sizeof(float2) + 2 * (size_t)N * sizeof(float)) +
                                     (size_t)nr * N));
    return;
  }
  // sum of sigma over the task's rows per load and component, rows combined in FP64
  if (threadIdx.x < nal * NP) {
    const int la = threadIdx.x / NP, k = threadIdx.x - la * NP;
    double acc = 0.0;
    for (int r = 0; r < nr; ++r) {
      if (EM) {  // sigma = (tau + u) / 2
        acc += 0.5 * ((double)sh.dc[la][1][r][k] + (double)N * (double)sh.dc[la][0][r][k]);
        continue;
      }
      const double tr = (double)sh.dc[la][0][r][0] + (double)sh.dc[la][0][r][1] + (double)sh.dc[la][0][r][2];
      const double se = (double)N * (2.0 * c.mu0 * (double)sh.dc[la][0][r][k] + (k < 3 ? c.lam0 * tr : 0.0));
      acc += (double)sh.dc[la][1][r][k] + se;
    }
    A.partR[((size_t)task * A.L + sh.al[la]) * NP + k] = acc;
  }
  if (threadIdx.x == 0)
    atomicAdd(A.bytes + HOM_K_ROW,
              (unsigned long long)(2 * (size_t)nr * nal * NP * H * sizeof(float2) + (size_t)nr * N));
}

// L2 prefetch of the first active load of row task `task` (every pair's rows, contiguous).
template <bool OUT>
__device__ __forceinline__ void prefetch_row3_task(const SolveArgs& A, int task) {
  const TaskR t = A.tR[task];
  const CellDev c = A.cells[t.cell];
  int l = -1;
  for (int q = 0; q < A.L && l < 0; ++q)
    if (OUT || A.active[t.cell * A.L + q]) l = q;
  if (l < 0) return;
  const float4* e = static_cast<const float4*>(A.eps[OUT ? (A.iters[t.cell * A.L + l] & 1) : (*A.it_dev & 1)]);
  const int z = t.row0 / c.n, y0 = t.row0 - z * c.n;
  const int P = (c.n / 2 + 2) / 2;
  for (int p = threadIdx.x; p < P; p += kT3)
    prefetch_l2(e + idx3(c, c.n, l, p, z, y0), (unsigned)(t.nrows * NP * sizeof(float4)));
}

// One CTA per task; CTA b prefetches the first load of task b + ahead (about the task that starts
// when this CTA ends: `ahead` CTAs are resident at once) into L2.
template <bool OUT, bool SRC, bool EM = false>
__global__ void __launch_bounds__(kT3, kMinB3) k_row_f3d(SolveArgs A, int ntasks, int ahead) {
  HOM_DBG_POISON();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ RowShared3 sh;
  float4* s = reinterpret_cast<float4*>(smem_raw);
  const int task = blockIdx.x;
  if (task + ahead < ntasks) prefetch_row3_task<OUT>(A, task + ahead);
  const TaskR t = A.tR[task];
  const CellDev c = A.cells[t.cell];
  // debug builds: the task's rows lie in one z plane of the cell
  if (!HOM_CHECK(A, t.row0 >= 0 && t.nrows >= 1 && t.row0 + t.nrows <= c.nrows &&
                        t.row0 / c.n == (t.row0 + t.nrows - 1) / c.n && t.load < A.L, (size_t)task))
    return;
  const FastPlanDev fp = A.fplans[c.fplan];
  switch (c.n) {
    case 27: row3_body<27, OUT, SRC, EM>(A, task, t, c, fp, s, sh); break;
    case 45: row3_body<45, OUT, SRC, EM>(A, task, t, c, fp, s, sh); break;
    case 81: row3_body<81, OUT, SRC, EM>(A, task, t, c, fp, s, sh); break;
    case 135: row3_body<135, OUT, SRC, EM>(A, task, t, c, fp, s, sh); break;
    case 243: row3_body<243, OUT, SRC, EM>(A, task, t, c, fp, s, sh); break;
    default: break;
  }
}

#ifndef HOM_3D_BULK
#define HOM_3D_BULK 1  // y passes: the tile in and out by bulk copies of one position each
#endif
#ifndef HOM_3D_GREEN_GPF
#define HOM_3D_GREEN_GPF 1  // Green pass: L2 prefetch of the task's own g (or u_hat) block before its forward FFT
#endif
#ifndef HOM_3D_GREEN_BULK
#define HOM_3D_GREEN_BULK 0  // the same for the Green pass, whose positions are a z plane apart in HBM
#endif

// Bulk copies of the N positions of a tile (NP float4 each, contiguous in HBM at stride gs float4,
// at stride SP in shared memory) in or out; threads issue one position each in turn.  `load`
// waits (bounded) for all of them on `bar`, initialised here; running out is recorded in A.dbg.
template <int N>
__device__ __forceinline__ void tile_bulk_load(const SolveArgs& A, float4* s, const float4* g, size_t gs,
                                               unsigned long long* bar) {
  fence_proxy_async();
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"((unsigned)(N * NP * sizeof(float4)))
                 : "memory");
  }
  __syncthreads();
  for (int p = threadIdx.x; p < N; p += kT3)
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(s + (size_t)p * SP)),
                 "l"(g + (size_t)p * gs), "r"((unsigned)(NP * sizeof(float4))), "r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tile_bulk_wait(const SolveArgs& A, unsigned long long* bar) {
  if (!mbar_wait(bar, 0, 1 << 22) && A.dbg) atomicCAS(A.dbg, 0u, 0xFFFFFFFFu);
  __syncthreads();
  if (threadIdx.x == 0) mbar_inval(bar);
}
template <int N>
__device__ __forceinline__ void tile_bulk_store(float4* g, size_t gs, const float4* s) {
  fence_proxy_async();
  __syncthreads();
  bool any = false;
  for (int p = threadIdx.x; p < N; p += kT3) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(g + (size_t)p * gs),
                 "r"(smem_u32(s + (size_t)p * SP)), "r"((unsigned)(NP * sizeof(float4)))
                 : "memory");
    any = true;
  }
  if (any) {
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    bulk_store_wait_read();
  }
}

// ------------------------------------------------------------------ y passes
// FWD: tau -> forward y-DFT -> tau (digit-reversed y positions).  Inverse: tau -> inverse y-DFT
// -> the next eps buffer (natural order).  One contiguous tile per task: [y][component].
template <int N, bool FWD>
__device__ __forceinline__ void ypass3_body(const SolveArgs& A, const TaskL& t, const CellDev& c,
                                            const FastPlanDev& fp, float4* s) {
  if (!A.active[t.cell * A.L + t.load]) return;
  const int it = *A.it_dev;
  const size_t tb = idx3(c, N, t.load, t.kx0 / 2, t.fixed, 0);
  const float4* in = static_cast<const float4*>(A.tau) + tb;
  float4* out = static_cast<float4*>(FWD ? A.tau : A.eps[(it + 1) & 1]) + tb;
  float2* tws = reinterpret_cast<float2*>(s + N * SP);
#if HOM_3D_BULK
  __shared__ __align__(8) unsigned long long ybar;
  tile_bulk_load<N>(A, s, in, NP, &ybar);
#else
  for (int i = threadIdx.x; i < N * NP; i += kT3) cp16(s + (i / NP) * SP + i % NP, in + i);
#endif
  for (int i = threadIdx.x; i < (N + 1) / 2; i += kT3) cp16(tws + 2 * i, fp.tw2 + 2 * i);
  cp_commit();
  cp_wait_all();
#if HOM_3D_BULK
  tile_bulk_wait(A, &ybar);
#endif
  __syncthreads();
  if (FWD) fft_dif_p<NP, N, true, float2, SP, kT3>(s, tws);
  else fft_dit_p<NP, N, false, float2, SP, kT3>(s, tws);
#if HOM_3D_BULK
  tile_bulk_store<N>(out, NP, s);
#else
  for (int i = threadIdx.x; i < N * NP; i += kT3) out[i] = s[(i / NP) * SP + i % NP];
#endif
  if (threadIdx.x == 0) {
    const int ntk = t.kx0 + 1 < c.H ? 2 : 1;
    atomicAdd(A.bytes + (FWD ? HOM_K_YFWD : HOM_K_YINV), (unsigned long long)(2 * (size_t)N * ntk * NP * sizeof(float2)));
  }
}

template <bool FWD>
__global__ void __launch_bounds__(kT3, 1024 / kT3) k_ypass_f3d(SolveArgs A) {
  HOM_DBG_POISON();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float4* s = reinterpret_cast<float4*>(smem_raw);
  const TaskL t = A.tY[blockIdx.x];
  const CellDev c = A.cells[t.cell];
  if (!HOM_CHECK(A, t.kx0 >= 0 && (t.kx0 & 1) == 0 && t.kx0 < c.H && t.fixed >= 0 && t.fixed < c.n &&
                        t.load >= 0 && t.load < A.L, (size_t)blockIdx.x))
    return;
  const FastPlanDev fp = A.fplans[c.fplan];
  switch (c.n) {
    case 27: ypass3_body<27, FWD>(A, t, c, fp, s); break;
    case 45: ypass3_body<45, FWD>(A, t, c, fp, s); break;
    case 81: ypass3_body<81, FWD>(A, t, c, fp, s); break;
    case 135: ypass3_body<135, FWD>(A, t, c, fp, s); break;
    case 243: ypass3_body<243, FWD>(A, t, c, fp, s); break;
    default: break;
  }
}

// ------------------------------------------------------------------ Green pass (z lines)
// Eyre-Milton scheme: the positions of one thread, lane by lane through em_core (hom_em.cuh); the
// private state is u_hat of the current iterate, [z position][6 components] as lane pairs (the
// layout of the tile), in place of g.
template <int N>
__device__ __forceinline__ void green3_em(int kx0, bool hasB, int py, const CellDev& c, const float* sx,
                                          const FastPlanDev& fp, float4* s, float4* ub, const double* Eld,
                                          Acc<float> (&acc)[3]) {
  CellConst<float> cc;
  cell_const(c, cc);
  const float nvT = (float)c.nv, inv_nv = cc.inv_nv, lam0 = cc.lam0, mu2_0 = cc.mu2;
  const float a0 = cc.lam0 / (cc.mu2 + 3.f * cc.lam0), inv_mu2_0 = 0.5f * cc.inv_mu0;
  const float X[2] = {__ldg(fp.xinat + kx0), hasB ? __ldg(fp.xinat + kx0 + 1) : 0.f}, Y = sx[py];
  float* sf = reinterpret_cast<float*>(s);
  float* uf = reinterpret_cast<float*>(ub);  // lane pairs, like the tile: [position][component]
  // one (position, lane) per item: lane h reads and writes its own floats of the lane pairs
  for (int i = threadIdx.x; i < 2 * N; i += kT3) {
    const int pos = i >> 1, h = i & 1;
    if (h && !hasB) continue;
    float2 th[NP], uh[NP], un[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      const float* T = sf + 4 * (pos * SP + k);
      const float* U = uf + 4 * (NP * pos + k);
      th[k] = make_float2(T[h], T[2 + h]);
      uh[k] = make_float2(U[h], U[2 + h]);
    }
    const float xi[3] = {X[h], Y, sx[pos]};
    em_core<float, 3>(th, uh, un, xi, h == 0 && kx0 == 0 && py == 0 && pos == 0, false, h == 0 && kx0 == 0, nvT,
                      inv_nv, lam0, mu2_0, a0, inv_mu2_0, cc.inv_mu0, cc.ratio, Eld, acc[0], acc[1], acc[2]);
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      float* T = sf + 4 * (pos * SP + k);
      float* U = uf + 4 * (NP * pos + k);
      T[h] = un[k].x;
      T[2 + h] = un[k].y;
      U[h] = un[k].x;
      U[2 + h] = un[k].y;
    }
  }
  if (!hasB)  // the missing lane B of the last pair stays zero
    for (int i = threadIdx.x; i < N * NP; i += kT3) {
      const int pos = i / NP, k = i - pos * NP;
      sf[4 * (pos * SP + k) + 1] = 0.f;
      sf[4 * (pos * SP + k) + 3] = 0.f;
    }
}

template <int N, bool EM = false>
__device__ __forceinline__ void green3_body(const SolveArgs& A, const TaskL& t, const CellDev& c,
                                            const FastPlanDev& fp, float4* s) {
  constexpr int H = (N + 1) / 2;
  const int cl = t.cell * A.L + t.load;
  if (!A.active[cl]) return;
  const int kx0 = t.kx0, py = t.fixed, p = kx0 / 2;
  const bool hasB = kx0 + 1 < H;
  float4* st = static_cast<float4*>(A.tau);
  const size_t zs = (size_t)N * NP;  // float4 stride between z planes at fixed y
  const size_t b0 = idx3(c, N, t.load, p, 0, py);
  float2* tws = reinterpret_cast<float2*>(s + N * SP);
  float* sx = reinterpret_cast<float*>(s + N * SP + (N + 1) / 2);
#if HOM_3D_GREEN_BULK
  __shared__ __align__(8) unsigned long long gbar;
  tile_bulk_load<N>(A, s, st + b0, zs, &gbar);
#else
  for (int i = threadIdx.x; i < N * NP; i += kT3) {
    const int zz = i / NP, k = i - zz * NP;
    cp16(s + zz * SP + k, st + b0 + zz * zs + k);
  }
#endif
  for (int i = threadIdx.x; i < (N + 1) / 2; i += kT3) cp16(tws + 2 * i, fp.tw2 + 2 * i);
  for (int i = threadIdx.x; i < (N + 3) / 4; i += kT3) cp16(sx + 4 * i, fp.xipos + 4 * i);
  cp_commit();
  cp_wait_all();
#if HOM_3D_GREEN_BULK
  tile_bulk_wait(A, &gbar);
#endif
  __syncthreads();
#if HOM_3D_GREEN_GPF
  // the private state of this (kx pair, ky) (contiguous: N positions x 3 or 6 float4) -> L2
  if (threadIdx.x < 32) {
    const size_t per = EM ? 6 : 3;
    const char* gsrc = reinterpret_cast<const char*>(
        static_cast<const float4*>(A.g) + (c.g_off + (((size_t)t.load * (c.Hp / 2) + p) * N + py) * (size_t)N * 2 * per) / 2);
    const unsigned bytes = (unsigned)(N * per * sizeof(float4));
    constexpr unsigned kPiece = 4096;
    for (unsigned o = threadIdx.x * kPiece; o < bytes; o += 32 * kPiece) prefetch_l2(gsrc + o, min(kPiece, bytes - o));
  }
#endif
  fft_dif_p<NP, N, true, float2, SP, kT3>(s, tws);  // forward: bin kz at position perm(kz)

  if constexpr (EM) {
    float4* ub = static_cast<float4*>(A.g) +
                 (c.g_off + (((size_t)t.load * (c.Hp / 2) + p) * N + py) * (size_t)N * 12) / 2;
    Acc<float> acc[3];
    green3_em<N>(kx0, hasB, py, c, sx, fp, s, ub, A.E + (size_t)cl * NP, acc);
    double tot[3];
    block_sum<float, 3, kT3>(acc, tot);  // contains the barrier before the inverse transform
    if (threadIdx.x == 0) {
      A.partC[2 * (size_t)blockIdx.x] = tot[0];
      A.partC[2 * (size_t)blockIdx.x + 1] = tot[1];
      A.partE[blockIdx.x] = tot[2];
    }
    fft_dit_p<NP, N, false, float2, SP, kT3>(s, tws);  // inverse: natural z order
#if HOM_3D_GREEN_BULK
    tile_bulk_store<N>(st + b0, zs, s);
#else
    for (int i = threadIdx.x; i < N * NP; i += kT3) {
      const int zz = i / NP, k = i - zz * NP;
      st[b0 + zz * zs + k] = s[zz * SP + k];
    }
#endif
    if (threadIdx.x == 0) {
      const int ntk = hasB ? 2 : 1;
      atomicAdd(A.bytes + HOM_K_GREEN, (unsigned long long)(4 * (size_t)N * ntk * NP * sizeof(float2)));
    }
    return;
  }

  CellConst<float> cc;
  cell_const(c, cc);
  const float2 mu0 = f2(0.5f * cc.mu2), lpm = f2(cc.lpm), ratio = f2(cc.ratio), inv_mu0 = f2(cc.inv_mu0);
  const float inv_nv = cc.inv_nv;
  const float rs2 = 0.707106781186547524400844362105f;
  const float2 X = make_float2(__ldg(fp.xinat + kx0), hasB ? __ldg(fp.xinat + kx0 + 1) : 0.f);
  const float2 Y = f2(sx[py]);
  const float2 XY2 = fma2(Y, Y, mul2(X, X));
  const float2 wgt = make_float2(kx0 == 0 ? 1.f : 2.f, hasB ? 2.f : 0.f);
  // g of this (kx pair, y position): [z position][3 lane pairs]
  float4* gb = static_cast<float4*>(A.g) +
               (c.g_off + (((size_t)t.load * (c.Hp / 2) + p) * N + py) * (size_t)N * 6) / 2;
  const double* Eld = A.E + (size_t)cl * NP;
  float2 r2s = make_float2(0.f, 0.f), r2c = r2s, rns = r2s, rnc = r2s;
  for (int pos = threadIdx.x; pos < N; pos += kT3) {
    const float2 Z = f2(sx[pos]);
    P2 T[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) T[k] = ldp(s[pos * SP + k]);
    P2 G[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) G[d] = ldp(gb[3 * pos + d]);
    // tau_hat as a tensor: t01 = T5 / sqrt 2, t02 = T4 / sqrt 2, t12 = T3 / sqrt 2
    const P2 t12 = scale(rs2, T[3]), t02 = scale(rs2, T[4]), t01 = scale(rs2, T[5]);
    auto dot3 = [&](const P2& a, const P2& b, const P2& cz) {  // X a + Y b + Z c
      return P2{fma2(Z, cz.re, fma2(Y, b.re, mul2(X, a.re))), fma2(Z, cz.im, fma2(Y, b.im, mul2(X, a.im)))};
    };
    const P2 V0 = dot3(T[0], t01, t02);
    const P2 V1 = dot3(t01, T[1], t12);
    const P2 V2 = dot3(t02, t12, T[2]);
    const float2 q2 = fma2(Z, Z, XY2);
    const P2 XG = dot3(G[0], G[1], G[2]);
    const P2 XV = dot3(V0, V1, V2);
    // residual r = tau_hat xi - K0 g, K0 g = mu0 q2 g + (lam0 + mu0) xi (xi . g)
    const float2 mq = mul2(mu0, q2);
    const float2 lx = mul2(lpm, X), ly = mul2(lpm, Y), lz = mul2(lpm, Z);
    auto resid = [&](const P2& V, const P2& Gd, float2 lxi) {
      return P2{sub2(sub2(V.re, mul2(mq, Gd.re)), mul2(lxi, XG.re)), sub2(sub2(V.im, mul2(mq, Gd.im)), mul2(lxi, XG.im))};
    };
    const P2 R0 = resid(V0, G[0], lx), R1 = resid(V1, G[1], ly), R2 = resid(V2, G[2], lz);
    float2 r2 = mul2(R0.re, R0.re);
    r2 = fma2(R0.im, R0.im, r2);
    r2 = fma2(R1.re, R1.re, r2);
    r2 = fma2(R1.im, R1.im, r2);
    r2 = fma2(R2.re, R2.re, r2);
    r2 = fma2(R2.im, R2.im, r2);
    const bool k0 = kx0 == 0 && py == 0 && pos == 0;  // k = 0: eps_hat(0) = E, g = 0, no residual
    const float2 iq = make_float2(k0 ? 0.f : __fdividef(1.f, q2.x), hasB ? __fdividef(1.f, q2.y) : 0.f);
    // g' = K0^-1 (tau_hat xi), eps_hat' = -sym(xi (x) g') / N_v
    const float2 imq = mul2(inv_mu0, iq);
    const float2 rq = mul2(ratio, iq);
    auto wvec = [&](const P2& V, float2 xi) {
      const float2 rxi = mul2(rq, xi);
      return P2{mul2(imq, sub2(V.re, mul2(rxi, XV.re))), mul2(imq, sub2(V.im, mul2(rxi, XV.im)))};
    };
    const P2 W0 = wvec(V0, X), W1 = wvec(V1, Y), W2 = wvec(V2, Z);
    const float2 nx = mul2(X, f2(-inv_nv)), ny = mul2(Y, f2(-inv_nv)), nz = mul2(Z, f2(-inv_nv));
    const float2 ns = f2(-rs2 * inv_nv);
    auto sym = [&](const P2& wa, float2 xb, const P2& wb, float2 xa) {  // -(xa wb + xb wa) / (sqrt2 N_v)
      return P2{mul2(ns, fma2(xa, wb.re, mul2(xb, wa.re))), mul2(ns, fma2(xa, wb.im, mul2(xb, wa.im)))};
    };
    P2 E[NP];
    E[0] = P2{mul2(nx, W0.re), mul2(nx, W0.im)};
    E[1] = P2{mul2(ny, W1.re), mul2(ny, W1.im)};
    E[2] = P2{mul2(nz, W2.re), mul2(nz, W2.im)};
    E[3] = sym(W1, Z, W2, Y);  // 23
    E[4] = sym(W0, Z, W2, X);  // 13
    E[5] = sym(W0, Y, W1, X);  // 12
    P2 Gn[3] = {W0, W1, W2};
    float2 wr = wgt;
    if (k0) {
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        E[k].re.x = (float)Eld[k];
        E[k].im.x = 0.f;
      }
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        Gn[d].re.x = 0.f;
        Gn[d].im.x = 0.f;
      }
      wr.x = 0.f;
    }
#pragma unroll
    for (int k = 0; k < NP; ++k) s[pos * SP + k] = stp(E[k]);
#pragma unroll
    for (int d = 0; d < 3; ++d) gb[3 * pos + d] = stp(Gn[d]);
    const float2 a1 = mul2(wr, r2), a2 = mul2(a1, iq);
    {
      const float2 yv = sub2(a1, r2c), tv = add2(r2s, yv);
      r2c = sub2(sub2(tv, r2s), yv);
      r2s = tv;
    }
    {
      const float2 yv = sub2(a2, rnc), tv = add2(rns, yv);
      rnc = sub2(sub2(tv, rns), yv);
      rns = tv;
    }
  }
  {
    Acc<float> vv[2];
    vv[0].s = r2s.x;
    vv[0].c = r2c.x;
    vv[0].add(r2s.y);
    vv[0].add(-r2c.y);
    vv[1].s = rns.x;
    vv[1].c = rnc.x;
    vv[1].add(rns.y);
    vv[1].add(-rnc.y);
    double tot[2];
    block_sum<float, 2, kT3>(vv, tot);  // contains the barrier before the inverse transform
    if (threadIdx.x == 0) {
      A.partC[2 * (size_t)blockIdx.x] = tot[0];
      A.partC[2 * (size_t)blockIdx.x + 1] = tot[1];
    }
  }
  fft_dit_p<NP, N, false, float2, SP, kT3>(s, tws);  // inverse: natural z order
#if HOM_3D_GREEN_BULK
  tile_bulk_store<N>(st + b0, zs, s);
#else
  for (int i = threadIdx.x; i < N * NP; i += kT3) {
    const int zz = i / NP, k = i - zz * NP;
    st[b0 + zz * zs + k] = s[zz * SP + k];
  }
#endif
  if (threadIdx.x == 0) {
    const int ntk = hasB ? 2 : 1;
    atomicAdd(A.bytes + HOM_K_GREEN,
              (unsigned long long)(2 * (size_t)N * ntk * NP * sizeof(float2) + 2 * (size_t)N * ntk * 3 * sizeof(float2)));
  }
}

template <bool EM = false>
__global__ void __launch_bounds__(kT3, kMinB3) k_green_f3d(SolveArgs A) {
  HOM_DBG_POISON();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float4* s = reinterpret_cast<float4*>(smem_raw);
  const TaskL t = A.tC[blockIdx.x];
  const CellDev c = A.cells[t.cell];
  if (!HOM_CHECK(A, t.kx0 >= 0 && (t.kx0 & 1) == 0 && t.kx0 < c.H && t.fixed >= 0 && t.fixed < c.n &&
                        t.load >= 0 && t.load < A.L, (size_t)blockIdx.x))
    return;
  const FastPlanDev fp = A.fplans[c.fplan];
  switch (c.n) {
    case 27: green3_body<27, EM>(A, t, c, fp, s); break;
    case 45: green3_body<45, EM>(A, t, c, fp, s); break;
    case 81: green3_body<81, EM>(A, t, c, fp, s); break;
    case 135: green3_body<135, EM>(A, t, c, fp, s); break;
    case 243: green3_body<243, EM>(A, t, c, fp, s); break;
    default: break;
  }
}

// eps = E: the stored x-spectrum holds E at kx = 0 (lane A of pair 0) of every row, zero elsewhere.
// EM: u = 2 c0 : E instead, and its 1/N_v-scaled spectrum at k = 0 in the Green pass's private state
// (pair 0, ky = 0, position 0, lane A; the rest is cleared by the caller).
template <bool EM = false>
__global__ void k_init_f3d(SolveArgs A, int ncells) {
  for (int cell = blockIdx.y; cell < ncells; cell += gridDim.y) {
    const CellDev c = A.cells[cell];
    const long long items = (long long)A.L * c.nrows * NP;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < items; i += (long long)gridDim.x * blockDim.x) {
      const int k = (int)(i % NP);
      const long long r = i / NP;
      const int row = (int)(r % c.nrows);
      const int l = (int)(r / c.nrows);
      const int z = row / c.n, y = row - z * c.n;
      const double* El = A.E + ((size_t)cell * A.L + l) * NP;
      double v = El[k];
      if (EM) {
        v = 2.0 * (2.0 * c.mu0 * El[k] + (k < 3 ? c.lam0 * (El[0] + El[1] + El[2]) : 0.0));
        if (row == 0)
          static_cast<float4*>(A.g)[(c.g_off + (size_t)l * (c.Hp / 2) * c.n * c.n * 12) / 2 + k] =
              make_float4((float)v, 0.f, 0.f, 0.f);
      }
      static_cast<float4*>(A.eps[0])[idx3(c, c.n, l, 0, z, y) + k] = make_float4((float)v, 0.f, 0.f, 0.f);
    }
  }
}

template <typename K>
int opt_in3(K kernel, size_t bytes) {
  if (bytes > 48 * 1024) HOM_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  return HOM_OK;
}

}  // namespace

bool fast3d_size(int n) {
  for (int k : kSizes3)
    if (k == n) return true;
  return false;
}

// row: tile | one-byte labels of 4 rows | twiddles | spare landing slots | per-phase constants;
// y: tile | twiddles;
// Green: tile | twiddles | wave numbers
size_t fast3d_smem_row(int nmax, int nphase_cell) {
  return (size_t)nmax * SP * sizeof(float4) + (size_t)kFastRows * ((nmax + 15) / 16 * 16) +
         ((size_t)nmax + 1) / 2 * 16 + (size_t)kRowSpare3 * sizeof(float4) + ((size_t)nphase_cell * 16 + 15) / 16 * 16;
}
size_t fast3d_smem_y(int nmax) { return (size_t)nmax * SP * sizeof(float4) + ((size_t)nmax + 1) / 2 * 16; }
size_t fast3d_smem_green(int nmax) {
  return (size_t)nmax * SP * sizeof(float4) + ((size_t)nmax + 1) / 2 * 16 + ((size_t)nmax + 3) / 4 * 16;
}

int fast3d_row(const SolveArgs& A, unsigned ntasks, size_t smem, bool out, cudaStream_t st) {
  int rc;
  if (A.scheme == HOM_SCHEME_EYRE_MILTON && out) {
    if ((rc = opt_in3(k_row_f3d<true, false, true>, smem)) != HOM_OK) return rc;
    k_row_f3d<true, false, true><<<ntasks, kT3, smem, st>>>(A, (int)ntasks,
                                                            resident_ctas(k_row_f3d<true, false, true>, kT3, smem));
  } else if (A.scheme == HOM_SCHEME_EYRE_MILTON) {
    if ((rc = opt_in3(k_row_f3d<false, false, true>, smem)) != HOM_OK) return rc;
    k_row_f3d<false, false, true><<<ntasks, kT3, smem, st>>>(A, (int)ntasks,
                                                             resident_ctas(k_row_f3d<false, false, true>, kT3, smem));
  } else if (out) {
    if ((rc = opt_in3(k_row_f3d<true, false>, smem)) != HOM_OK) return rc;
    k_row_f3d<true, false><<<ntasks, kT3, smem, st>>>(A, (int)ntasks, resident_ctas(k_row_f3d<true, false>, kT3, smem));
  } else if (A.src) {  // adjoint solve: the constitutive step takes the source term
    if ((rc = opt_in3(k_row_f3d<false, true>, smem)) != HOM_OK) return rc;
    k_row_f3d<false, true><<<ntasks, kT3, smem, st>>>(A, (int)ntasks, resident_ctas(k_row_f3d<false, true>, kT3, smem));
  } else {
    if ((rc = opt_in3(k_row_f3d<false, false>, smem)) != HOM_OK) return rc;
    k_row_f3d<false, false><<<ntasks, kT3, smem, st>>>(A, (int)ntasks, resident_ctas(k_row_f3d<false, false>, kT3, smem));
  }
  return HOM_OK;
}

int fast3d_ypass(const SolveArgs& A, unsigned ntasks, size_t smem, bool fwd, cudaStream_t st) {
  int rc;
  if (fwd) {
    if ((rc = opt_in3(k_ypass_f3d<true>, smem)) != HOM_OK) return rc;
    k_ypass_f3d<true><<<ntasks, kT3, smem, st>>>(A);
  } else {
    if ((rc = opt_in3(k_ypass_f3d<false>, smem)) != HOM_OK) return rc;
    k_ypass_f3d<false><<<ntasks, kT3, smem, st>>>(A);
  }
  return HOM_OK;
}

int fast3d_green(const SolveArgs& A, unsigned ntasks, size_t smem, cudaStream_t st) {
  if (A.scheme == HOM_SCHEME_EYRE_MILTON) {
    int rc = opt_in3(k_green_f3d<true>, smem);
    if (rc != HOM_OK) return rc;
    k_green_f3d<true><<<ntasks, kT3, smem, st>>>(A);
    return HOM_OK;
  }
  int rc = opt_in3(k_green_f3d<false>, smem);
  if (rc != HOM_OK) return rc;
  k_green_f3d<false><<<ntasks, kT3, smem, st>>>(A);
  return HOM_OK;
}

int fast3d_init(const SolveArgs& A, int ncells, cudaStream_t st) {
  dim3 grid(64, (unsigned)std::min(ncells, 65535));
  if (A.scheme == HOM_SCHEME_EYRE_MILTON) k_init_f3d<true><<<grid, 256, 0, st>>>(A, ncells);
  else k_init_f3d<false><<<grid, 256, 0, st>>>(A, ncells);
  return HOM_OK;
}

}  // namespace hom

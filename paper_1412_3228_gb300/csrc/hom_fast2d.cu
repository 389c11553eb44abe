// Specialised FP32 row and Green passes of the 2D fixed-point scheme (section 2, eqs. 1-a, 1-b,
// 2) for grid sizes n with a radix plan fixed at compile time.
//
// Lane pairs.  Shared memory holds one float4 per (position, pair): (re_A, re_B, im_A, im_B), the
// same position of two complex lines A and B.  Every butterfly, the Green operator and the
// constitutive update then act on both lines with packed FP32x2 instructions (add/sub/mul/fma
// .f32x2), one instruction per pair of values.
//   row pass  : pair c = Mandel component c; line A = real rows y0 + i*(y0+1), line B = rows
//               y0+2 + i*(y0+3).  One CTA handles 4 rows and loops over the active loads.
//   Green pass: pair c = component c; line A = column kx0, line B = column kx0 + 1.
// With the three components side by side, the element stride is 48 bytes, so consecutive
// positions fall on distinct bank quads: the stage accesses are free of bank conflicts.
//
// Transforms are the in-place mixed-radix DIF (natural -> digit-reversed) and DIT (digit-reversed
// -> natural) of hom_common.cuh with the radices as template parameters: every index division is
// by a compile-time constant.  The row pass works on x samples at digit-reversed positions and
// reads one-byte labels permuted the same way (label8); the Green pass reads the wave number of each
// position from a table.
//
// State in HBM.  The specialised passes keep the mixed-domain state (eps buffers, tau) tiled by kx
// pairs (tile_index): one Green task reads one contiguous tile with 16-byte asynchronous copies
// straight into its shared-memory layout, and a row task reads 192 contiguous bytes per pair.  The
// Green pass keeps its displacement-like state g as [load][column pair][position][4 complex].
// Both layouts are private to these passes: the initial state and the output fields are written
// by the kernels here.
#define HOM_FILE_ID 2
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "hom_fast2d.h"
#include "hom_plan.h"
#include "hom_solve_args.cuh"
#include "hom_fastfft.cuh"
#include "hom_em.cuh"

namespace hom {
namespace {

#ifndef HOM_GREEN_TW2
#define HOM_GREEN_TW2 1  // Green pass with a scalar twiddle table (three CTAs per SM)
#endif
#ifndef HOM_ROW_TW2
#define HOM_ROW_TW2 1    // row pass with a scalar twiddle table (three CTAs per SM)
#endif
#ifndef HOM_ROW_LANDING
#define HOM_ROW_LANDING 1  // row pass: rows land by cp.async in their line slots (0: register loads)
#endif
#ifndef HOM_ROW_PREFETCH
#define HOM_ROW_PREFETCH 0  // row pass L2 prefetch: 1 = the next load, 2 = the next task (bit mask)
#endif
#ifndef HOM_GREEN_BULK
#define HOM_GREEN_BULK 1  // Green pass: its contiguous tile in and out by one bulk copy each (TMA unit)
#endif
#ifndef HOM_GREEN_GPF
#define HOM_GREEN_GPF 1  // Green pass: L2 prefetch of the task's own g (or u_hat) block before its forward FFT
#endif
#ifndef HOM_GREEN_PREFETCH
#define HOM_GREEN_PREFETCH 0  // Green pass: L2 prefetch of the task that starts next
#endif
constexpr int NP = 3;  // lane pairs per position (2D Mandel components)
constexpr int kFastSizes[] = {45, 75, 135, 225, 405, 1215};  // sizes with specialised 2D passes

// ------------------------------------------------------------------ state layout
// The mixed-domain state of a cell (eps buffers and tau) is tiled by kx pairs: for load l, pair
// p = kx / 2 (T = Hp / 2 pairs) and row y, the three components are float4 lane pairs
// (re(kx = 2p), re(2p + 1), im(2p), im(2p + 1)).  A Green-pass task reads and writes one
// contiguous tile of n rows; a row-pass task reads 4 consecutive rows of every pair (192 bytes).
__device__ __forceinline__ size_t tile_index(const CellDev& c, int n, int l, int p, int y) {
  return (size_t)c.ws_off / 2 + (((size_t)l * (c.Hp / 2) + p) * n + y) * NP;
}

constexpr uint32_t kLabel8Mixed = 255;  // one-byte label of a mixed voxel

constexpr int kRowSpare = 2 * NP * kFastRows;  // float4 entries of the row pass's spare landing area
template <int N>
__device__ __forceinline__ float4* row_slot(float4* s, float4* spare, int p, int k, int r) {
  return row_slot_p<N, NP, NP>(s, spare, p, k, r);
}

// ------------------------------------------------------------------ row pass
// eps (stored x half-spectra) -> inverse x-DFT -> tau = sigma - c0 : eps -> forward x-DFT -> tau.
// OUT: the final fields eps and sigma of the returned iterate (real, solver output layout).
struct RowShared {
  int al[kMaxLoads], nal;                    // active loads
  float dc[kMaxLoads][2][kFastRows][NP];     // [load][eps row mean, tau row sum][row][comp]
};

// EM (Eyre-Milton scheme): the stored state is u = sigma + c0 : eps.  A pure voxel's tau is then
// W u with the isotropic W = (c - c0)(c + c0)^-1 (a per-phase pair of constants in place of
// (lam - lam0, 2 mu - 2 mu0)); a mixed group first solves eps = (c~ + c0)^-1 u per voxel and takes
// tau = c~ : eps - c0 : eps; the output pass turns u into eps first; the row sums of sigma are
// (tau + u) / 2.
template <int N, bool OUT, bool SRC, bool EM = false>
__device__ __forceinline__ void row_body(const SolveArgs& A, int task, const TaskR& t, const CellDev& c,
                                         const FastPlanDev& fp, float4* s, RowShared& sh) {
  constexpr int H = (N + 1) / 2;
  constexpr int P = (H + 1) / 2;  // kx pairs holding data
  int* s_al = sh.al;
  int& s_nal = sh.nal;
  auto& s_dc = sh.dc;
  const int it = *A.it_dev;
  if (threadIdx.x == 0) {
    int nal = 0;
    for (int l = 0; l < A.L; ++l) {
      const int cl = t.cell * A.L + l;
      if ((t.load < 0 || l == t.load) && (OUT || A.active[cl])) s_al[nal++] = l;
    }
    s_nal = nal;
  }
  __syncthreads();
  const int nal = s_nal;
  if (nal == 0) return;
  const int y0 = t.row0, nr = t.nrows;
  CellConst<float> cc;
  cell_const(c, cc);
  // OUT: sigma = c~ : eps, i.e. the update with a zero reference medium
  const float lam0 = OUT ? 0.f : cc.lam0, mu2_0 = OUT ? 0.f : cc.mu2;
  const float lam_em = cc.lam0, mu2_em = cc.mu2;  // EM: the reference medium of (c + c0)^-1, also when OUT
  float4* taub = static_cast<float4*>(A.tau);
  const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
  // one-byte labels of the task's rows (transform order) and the twiddle table -> shared memory,
  // behind the first loads
  constexpr int NL = (N + 15) / 16 * 16;  // label row stride (bytes)
  uint8_t* slab = reinterpret_cast<uint8_t*>(s + N * NP);
  {
    const uint4* src = reinterpret_cast<const uint4*>(A.label8 + c.lp_off + (size_t)y0 * NL);
    for (int i = threadIdx.x; i < nr * NL / 16; i += kT) cp16(slab + 16 * i, src + i);
  }
#if HOM_ROW_TW2
  float2* tws = reinterpret_cast<float2*>(s + N * NP + kFastRows * NL / 16);
  for (int i = threadIdx.x; i < (N + 1) / 2; i += kT) cp16(tws + 2 * i, fp.tw2 + 2 * i);
  float4* spare = s + N * NP + kFastRows * NL / 16 + (N + 1) / 2;
#else
  float4* tws = s + N * NP + kFastRows * NL / 16;
  for (int i = threadIdx.x; i < N; i += kT) cp16(tws + i, fp.tw4 + i);
  float4* spare = s + N * NP + kFastRows * NL / 16 + N;
#endif
  float2* sph = reinterpret_cast<float2*>(spare + kRowSpare);
  float2* sinv = sph + c.nph;  // EM: per local phase, (c + c0)^-1 as the pair (coefficient of tr(u) I, of u)
  cp_commit();
  // per local phase (lam - lam0, 2 mu - 2 mu0) for the pure-voxel update (visible after the next barrier)
  for (int i = threadIdx.x; i < c.nph; i += kT) {
    const float* pc = A.phase_c32 + (size_t)__ldg(A.cell_phases + c.ph_off + i) * 6;
    const float lam = __ldg(pc + 1);
    const float mu2 = __ldg(pc) - lam;
    sph[i] = make_float2(lam - lam0, mu2 - mu2_0);
    if (EM) {
      // (c + c0)^-1: volumetric eigenvalue 2 (lam + lam0) + (2 mu + 2 mu0), deviatoric 2 mu + 2 mu0
      const double l = (double)lam, m2 = (double)mu2, l0 = c.lam0, m20 = 2.0 * c.mu0;
      const double ms2 = m2 + m20, ks = 2.0 * (l + l0) + ms2;
      sinv[i] = make_float2((float)((1.0 / ks - 1.0 / ms2) * 0.5), (float)(1.0 / ms2));
      if (!OUT) {  // W = (c - c0)(c + c0)^-1: volumetric (k - k0)/(k + k0), deviatoric (2mu - 2mu0)/(2mu + 2mu0)
        const double aK = (m2 - m20) / ms2, aJ = (2.0 * (l - l0) + (m2 - m20)) / ks;
        sph[i] = make_float2((float)(0.5 * (aJ - aK)), (float)aK);
      }
    }
  }

  for (int la = 0; la < nal; ++la) {
    const int l = s_al[la];
    const float4* ein = static_cast<const float4*>(A.eps[OUT ? (A.iters[t.cell * A.L + l] & 1) : (it & 1)]);
#if HOM_ROW_LANDING
    // 1. four half-spectrum rows -> two Hermitian-extended complex lines per component.  Item
    // (p, k) = kx pair p, component k: its four row values (one 16-byte lane pair each) land, by
    // asynchronous copies all in flight at once, in the tile slots of the four line positions
    // they produce (row_slot), and are turned into line values in place below.  Rows beyond the
    // task (r >= nr) are zero-filled by the copy itself.
    for (int f = threadIdx.x; f < P * NP; f += kT) {
      const int p = f / NP, k = f - p * NP;
      const float4* src = ein + tile_index(c, N, l, p, y0) + k;
#pragma unroll
      for (int r = 0; r < kFastRows; ++r)
        cp16z(row_slot<N>(s, spare, p, k, r), src + (size_t)(r < nr ? r : 0) * NP, r < nr ? 16u : 0u);
    }
    cp_commit();
    // the next active load's rows of every pair (192 contiguous bytes each) -> L2, so that its
    // copies above hit L2 while this load's transforms run
    if ((HOM_ROW_PREFETCH & 1) && la + 1 < nal) {
      const float4* nx = static_cast<const float4*>(A.eps[OUT ? (A.iters[t.cell * A.L + s_al[la + 1]] & 1) : (it & 1)]);
      for (int p = threadIdx.x; p < P; p += kT)
        prefetch_l2(nx + tile_index(c, N, s_al[la + 1], p, y0), (unsigned)(nr * NP * sizeof(float4)));
    }
    cp_wait_all();
    __syncthreads();
    for (int f = threadIdx.x; f < P * NP; f += kT) {
      const int p = f / NP, k = f - p * NP;
      float4 v[kFastRows];
#pragma unroll
      for (int r = 0; r < kFastRows; ++r) v[r] = *row_slot<N>(s, spare, p, k, r);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int kx = 2 * p + h;
        if (kx >= H) break;
        // row r at kx: (re, im) = lane h of v[r]
        const float2 q0 = h ? make_float2(v[0].y, v[0].w) : make_float2(v[0].x, v[0].z);
        const float2 q1 = h ? make_float2(v[1].y, v[1].w) : make_float2(v[1].x, v[1].z);
        const float2 q2 = h ? make_float2(v[2].y, v[2].w) : make_float2(v[2].x, v[2].z);
        const float2 q3 = h ? make_float2(v[3].y, v[3].w) : make_float2(v[3].x, v[3].z);
        // A + iB at kx and conj(A) + i conj(B) at n - kx, for (A, B) = (row 0, row 1) and (row 2, row 3)
        s[kx * NP + k] = make_float4(q0.x - q1.y, q2.x - q3.y, q0.y + q1.x, q2.y + q3.x);
        if (kx > 0) {
          s[(N - kx) * NP + k] = make_float4(q0.x + q1.y, q2.x + q3.y, q1.x - q0.y, q3.x - q2.y);
        } else {
          s_dc[la][0][0][k] = q0.x;
          s_dc[la][0][1][k] = q1.x;
          s_dc[la][0][2][k] = q2.x;
          s_dc[la][0][3][k] = q3.x;
        }
      }
    }
    __syncthreads();
#else
    // 1. four half-spectrum rows -> two Hermitian-extended complex lines per component; item
    // (p, k) reads rows y0..y0+3 of pair p (U items per round: 4 U loads in flight per thread)
    constexpr int U = 1;
    for (int f0 = threadIdx.x; f0 < P * NP; f0 += U * kT) {
      float4 v[U][kFastRows];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int f = f0 + u * kT;
        const int p = f / NP, k = f - p * NP;
        const size_t b = tile_index(c, N, l, p, y0) + k;
#pragma unroll
        for (int r = 0; r < kFastRows; ++r) v[u][r] = (f < P * NP && r < nr) ? ein[b + (size_t)r * NP] : z4;
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int f = f0 + u * kT;
        if (f >= P * NP) continue;
        const int p = f / NP, k = f - p * NP;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int kx = 2 * p + h;
          if (kx >= H) break;
          // row r at kx: (re, im) = lane h of v[u][r]
          const float2 q0 = h ? make_float2(v[u][0].y, v[u][0].w) : make_float2(v[u][0].x, v[u][0].z);
          const float2 q1 = h ? make_float2(v[u][1].y, v[u][1].w) : make_float2(v[u][1].x, v[u][1].z);
          const float2 q2 = h ? make_float2(v[u][2].y, v[u][2].w) : make_float2(v[u][2].x, v[u][2].z);
          const float2 q3 = h ? make_float2(v[u][3].y, v[u][3].w) : make_float2(v[u][3].x, v[u][3].z);
          // A + iB at kx and conj(A) + i conj(B) at n - kx, for (A, B) = (row 0, row 1) and (row 2, row 3)
          s[kx * NP + k] = make_float4(q0.x - q1.y, q2.x - q3.y, q0.y + q1.x, q2.y + q3.x);
          if (kx > 0) {
            s[(N - kx) * NP + k] = make_float4(q0.x + q1.y, q2.x + q3.y, q1.x - q0.y, q3.x - q2.y);
          } else {
            s_dc[la][0][0][k] = q0.x;
            s_dc[la][0][1][k] = q1.x;
            s_dc[la][0][2][k] = q2.x;
            s_dc[la][0][3][k] = q3.x;
          }
        }
      }
    }
    cp_wait_all();
    __syncthreads();
#endif
    fft_dif_p<NP, N, false>(s, tws);  // inverse: eps at digit-reversed positions

    // 2. constitutive update: lanes (x, y, z, w) of a float4 are rows (0, 2, 1, 3).  A one-byte
    // label is the local phase index of a pure voxel, or kLabel8Mixed (full label read from the
    // material, which also covers any voxel whose phase is not in the cell's list).
    for (int pos = threadIdx.x; pos < N; pos += kT) {
      uint32_t lab[kFastRows];
      bool mixed = false;
#pragma unroll
      for (int r = 0; r < kFastRows; ++r) {
        lab[r] = r < nr ? (uint32_t)slab[r * NL + pos] : 0u;
        mixed |= lab[r] == kLabel8Mixed;
      }
      uint32_t loc[kFastRows];  // the one-byte labels (EM: per-phase constants of pure voxels)
#pragma unroll
      for (int r = 0; r < kFastRows; ++r) loc[r] = lab[r];
      if (mixed) {  // full labels: the material's for mixed voxels, global phases for the others
        const int x = __ldg(fp.iperm + pos);
#pragma unroll
        for (int r = 0; r < kFastRows; ++r)
          lab[r] = lab[r] == kLabel8Mixed ? __ldg(A.label + c.vox_off + (size_t)(y0 + r) * N + x)
                                          : (uint32_t)__ldg(A.cell_phases + c.ph_off + lab[r]);
      }
      float4 e[NP];
#pragma unroll
      for (int k = 0; k < NP; ++k) e[k] = s[pos * NP + k];
      if (EM && (OUT || mixed)) {
        // e holds u: eps = (c~ + c0)^-1 u, per voxel (mixed: the per-call table; pure: in closed form)
        float ev[NP][kFastRows];
#pragma unroll
        for (int r = 0; r < kFastRows; ++r) {
          float u[NP];
#pragma unroll
          for (int k = 0; k < NP; ++k) u[k] = r == 0 ? e[k].x : r == 1 ? e[k].z : r == 2 ? e[k].y : e[k].w;
          if (mixed && (lab[r] & HOM_MIXED_BIT)) {
            const float* M = static_cast<const float*>(A.em_minv) + (size_t)(lab[r] & ~HOM_MIXED_BIT) * 6;
            ev[0][r] = __ldg(M) * u[0] + __ldg(M + 1) * u[1] + __ldg(M + 2) * u[2];
            ev[1][r] = __ldg(M + 1) * u[0] + __ldg(M + 3) * u[1] + __ldg(M + 4) * u[2];
            ev[2][r] = __ldg(M + 2) * u[0] + __ldg(M + 4) * u[1] + __ldg(M + 5) * u[2];
          } else {
            float2 d;
            if (loc[r] == kLabel8Mixed) {  // a pure voxel whose phase is not in the cell's list (rare)
              const float* pc = A.phase_c32 + (size_t)lab[r] * 6;
              const float l = __ldg(pc + 1), m2 = __ldg(pc) - l;
              const float ms2 = m2 + mu2_em, ks = 2.f * (l + lam_em) + ms2;
              d = make_float2((1.f / ks - 1.f / ms2) * 0.5f, 1.f / ms2);
            } else {
              d = sinv[loc[r]];
            }
            const float tr = u[0] + u[1];
            ev[0][r] = d.y * u[0] + d.x * tr;
            ev[1][r] = d.y * u[1] + d.x * tr;
            ev[2][r] = d.y * u[2];
          }
        }
#pragma unroll
        for (int k = 0; k < NP; ++k) e[k] = make_float4(ev[k][0], ev[k][2], ev[k][1], ev[k][3]);
      }
      float4 o[NP];
      if (!mixed) {
        // pure voxels: tau = (lam - lam0) tr(eps) I + (2 mu - 2 mu0) eps
        float dl[kFastRows], dm[kFastRows];
#pragma unroll
        for (int r = 0; r < kFastRows; ++r) {
          const float2 d = sph[lab[r]];
          dl[r] = d.x;
          dm[r] = d.y;
        }
        const float2 dl_lo = make_float2(dl[0], dl[2]), dl_hi = make_float2(dl[1], dl[3]);
        const float2 dm_lo = make_float2(dm[0], dm[2]), dm_hi = make_float2(dm[1], dm[3]);
        const float2 tr_lo = add2(make_float2(e[0].x, e[0].y), make_float2(e[1].x, e[1].y));
        const float2 tr_hi = add2(make_float2(e[0].z, e[0].w), make_float2(e[1].z, e[1].w));
#pragma unroll
        for (int k = 0; k < NP; ++k) {
          float2 lo = mul2(dm_lo, make_float2(e[k].x, e[k].y));
          float2 hi = mul2(dm_hi, make_float2(e[k].z, e[k].w));
          if (k < 2) {
            lo = fma2(dl_lo, tr_lo, lo);
            hi = fma2(dl_hi, tr_hi, hi);
          }
          o[k] = make_float4(lo.x, lo.y, hi.x, hi.y);
        }
      } else {
        float out[NP][kFastRows];
#pragma unroll
        for (int r = 0; r < kFastRows; ++r) {
          float ev[NP];
#pragma unroll
          for (int k = 0; k < NP; ++k) ev[k] = r == 0 ? e[k].x : r == 1 ? e[k].z : r == 2 ? e[k].y : e[k].w;
          float C[6];
          const float* src = (lab[r] & HOM_MIXED_BIT) ? A.mixed_c32 + (size_t)(lab[r] & ~HOM_MIXED_BIT) * 6
                                                      : A.phase_c32 + (size_t)lab[r] * 6;
#pragma unroll
          for (int q = 0; q < 6; ++q) C[q] = __ldg(src + q);
          const float tr0 = ev[0] + ev[1];
          // packed upper triangle of the 3x3 Mandel matrix: (00, 01, 02, 11, 12, 22)
          const float sg0 = C[0] * ev[0] + C[1] * ev[1] + C[2] * ev[2];
          const float sg1 = C[1] * ev[0] + C[3] * ev[1] + C[4] * ev[2];
          const float sg2 = C[2] * ev[0] + C[4] * ev[1] + C[5] * ev[2];
          out[0][r] = sg0 - (mu2_0 * ev[0] + lam0 * tr0);
          out[1][r] = sg1 - (mu2_0 * ev[1] + lam0 * tr0);
          out[2][r] = sg2 - mu2_0 * ev[2];
        }
#pragma unroll
        for (int k = 0; k < NP; ++k) o[k] = make_float4(out[k][0], out[k][2], out[k][1], out[k][3]);
      }
      if constexpr (SRC) {
        // adjoint solve: the stiffness acts on w - S, so tau = (c~ - c0) : w - c~ : S, with the
        // source S (real field, solver output layout) read at the rows' voxels
        const int x = __ldg(fp.iperm + pos);
        const float* S = static_cast<const float*>(A.src) + c.fld_off + (size_t)l * NP * c.nv + (size_t)y0 * N + x;
        float cs[NP][kFastRows];
#pragma unroll
        for (int r = 0; r < kFastRows; ++r) {
#pragma unroll
          for (int k = 0; k < NP; ++k) cs[k][r] = 0.f;
          if (r >= nr) continue;
          const uint32_t L = mixed ? lab[r] : (uint32_t)__ldg(A.cell_phases + c.ph_off + lab[r]);
          const float* C = (L & HOM_MIXED_BIT) ? A.mixed_c32 + (size_t)(L & ~HOM_MIXED_BIT) * 6 : A.phase_c32 + (size_t)L * 6;
          float sv[NP];
#pragma unroll
          for (int k = 0; k < NP; ++k) sv[k] = __ldg(S + (size_t)k * c.nv + (size_t)r * N);
          cs[0][r] = __ldg(C) * sv[0] + __ldg(C + 1) * sv[1] + __ldg(C + 2) * sv[2];
          cs[1][r] = __ldg(C + 1) * sv[0] + __ldg(C + 3) * sv[1] + __ldg(C + 4) * sv[2];
          cs[2][r] = __ldg(C + 2) * sv[0] + __ldg(C + 4) * sv[1] + __ldg(C + 5) * sv[2];
        }
#pragma unroll
        for (int k = 0; k < NP; ++k)
          o[k] = make_float4(o[k].x - cs[k][0], o[k].y - cs[k][2], o[k].z - cs[k][1], o[k].w - cs[k][3]);
      }
      if (OUT) {
        // real fields of rows y0 + r at x = iperm[pos]
        const int x = __ldg(fp.iperm + pos);
        float* oe = static_cast<float*>(A.out_eps);
        float* os = static_cast<float*>(A.out_sig);
        const size_t base = c.fld_off + (size_t)l * NP * c.nv + (size_t)y0 * N + x;
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
        for (int k = 0; k < NP; ++k) s[pos * NP + k] = o[k];
      }
    }
    __syncthreads();  // the tile is read above and rewritten below (or by the next load's fill)
    if (OUT) continue;
    fft_dit_p<NP, N, true>(s, tws);  // forward: natural order

    // 3. split the two real rows of each line; store the half spectra of tau, pair by pair
    for (int f = threadIdx.x; f < P * NP; f += kT) {
      const int p = f / NP, k = f - p * NP;
      float4 w[kFastRows];  // rows 0..3 at (kx = 2p, 2p + 1): (re, re, im, im)
#pragma unroll
      for (int r = 0; r < kFastRows; ++r) w[r] = z4;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int kx = 2 * p + h;
        if (kx >= H) break;
        const float4 Z = s[kx * NP + k];
        const float4 Zm = s[(kx == 0 ? 0 : N - kx) * NP + k];
        // (Z[k] + conj Z[n-k]) / 2 -> first row of a line, (Z[k] - conj Z[n-k]) / 2i -> second row
        const float2 o0 = make_float2(0.5f * (Z.x + Zm.x), 0.5f * (Z.z - Zm.z));
        const float2 o1 = make_float2(0.5f * (Z.z + Zm.z), 0.5f * (Zm.x - Z.x));
        const float2 o2 = make_float2(0.5f * (Z.y + Zm.y), 0.5f * (Z.w - Zm.w));
        const float2 o3 = make_float2(0.5f * (Z.w + Zm.w), 0.5f * (Zm.y - Z.y));
        if (h == 0) {
          w[0].x = o0.x; w[0].z = o0.y; w[1].x = o1.x; w[1].z = o1.y;
          w[2].x = o2.x; w[2].z = o2.y; w[3].x = o3.x; w[3].z = o3.y;
          if (kx == 0) {
            s_dc[la][1][0][k] = o0.x;
            s_dc[la][1][1][k] = o1.x;
            s_dc[la][1][2][k] = o2.x;
            s_dc[la][1][3][k] = o3.x;
          }
        } else {
          w[0].y = o0.x; w[0].w = o0.y; w[1].y = o1.x; w[1].w = o1.y;
          w[2].y = o2.x; w[2].w = o2.y; w[3].y = o3.x; w[3].w = o3.y;
        }
      }
      const size_t b = tile_index(c, N, l, p, y0) + k;
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
                                     (size_t)nr * N * 4));
    return;
  }
  // sum of sigma over the task's rows per load and component (see the generic row pass):
  //   sum_x sigma = sum_x tau + c0 : (n * row mean of eps), rows combined in FP64
  if (threadIdx.x < nal * NP) {
    const int la = threadIdx.x / NP, k = threadIdx.x - la * NP;
    double acc = 0.0;
    for (int r = 0; r < nr; ++r) {
      if (EM) {  // sigma = (tau + u) / 2
        acc += 0.5 * ((double)s_dc[la][1][r][k] + (double)N * (double)s_dc[la][0][r][k]);
        continue;
      }
      const double tr = (double)s_dc[la][0][r][0] + (double)s_dc[la][0][r][1];
      const double se = (double)N * (2.0 * c.mu0 * (double)s_dc[la][0][r][k] + (k < 2 ? c.lam0 * tr : 0.0));
      acc += (double)s_dc[la][1][r][k] + se;
    }
    A.partR[((size_t)task * A.L + s_al[la]) * NP + k] = acc;
  }
  if (threadIdx.x == 0)
    atomicAdd(A.bytes + HOM_K_ROW,
              (unsigned long long)(2 * (size_t)nr * nal * NP * H * sizeof(float2) + (size_t)nr * N));
}

// L2 prefetch of the first active load of row task `task` (every pair's rows, 16 * 3 * nrows
// contiguous bytes each), issued while the CTA still works on its current task.
template <bool OUT>
__device__ __forceinline__ void prefetch_row_task(const SolveArgs& A, int task) {
  const TaskR t = A.tR[task];
  const CellDev c = A.cells[t.cell];
  int l = -1;
  for (int q = 0; q < A.L && l < 0; ++q)
    if (OUT || A.active[t.cell * A.L + q]) l = q;
  if (l < 0) return;
  const float4* e = static_cast<const float4*>(A.eps[OUT ? (A.iters[t.cell * A.L + l] & 1) : (*A.it_dev & 1)]);
  const int P = (c.n / 2 + 2) / 2;
  for (int p = threadIdx.x; p < P; p += kT)
    prefetch_l2(e + tile_index(c, c.n, l, p, t.row0), (unsigned)(t.nrows * NP * sizeof(float4)));
}

// One CTA per task.  `ahead` is the number of CTAs resident on the device at once: task b + ahead
// is about the one that starts when this CTA ends, so CTA b prefetches its first load into L2.
template <bool OUT, bool SRC, bool EM = false>
__global__ void __launch_bounds__(kT, HOM_ROW_TW2 ? 3 : 2) k_row_f2d(SolveArgs A, int ntasks, int ahead) {
  HOM_DBG_POISON();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ RowShared sh;
  float4* s = reinterpret_cast<float4*>(smem_raw);
  const int task = blockIdx.x;
  if ((HOM_ROW_PREFETCH & 2) && task + ahead < ntasks) prefetch_row_task<OUT>(A, task + ahead);
  const TaskR t = A.tR[task];
  const CellDev c = A.cells[t.cell];
  // debug builds: the task's rows lie in the cell (the CTA skips a bad task as a whole)
  if (!HOM_CHECK(A, t.row0 >= 0 && t.nrows >= 1 && t.nrows <= kFastRows && t.row0 + t.nrows <= c.nrows &&
                        t.load < A.L, (size_t)task))
    return;
  const FastPlanDev fp = A.fplans[c.fplan];
  switch (c.n) {
    case 45: row_body<45, OUT, SRC, EM>(A, task, t, c, fp, s, sh); break;
    case 75: row_body<75, OUT, SRC, EM>(A, task, t, c, fp, s, sh); break;
    case 135: row_body<135, OUT, SRC, EM>(A, task, t, c, fp, s, sh); break;
    case 225: row_body<225, OUT, SRC, EM>(A, task, t, c, fp, s, sh); break;
    case 405: row_body<405, OUT, SRC, EM>(A, task, t, c, fp, s, sh); break;
    case 1215: row_body<1215, OUT, SRC, EM>(A, task, t, c, fp, s, sh); break;
    default: break;
  }
}

// eps = E: the stored x-spectrum holds E at kx = 0 of every row (lane A of pair 0), zero elsewhere.
// EM: u = 2 c0 : E instead, and its 1/N_v-scaled spectrum at k = 0 in the Green pass's private state
// (pair 0, position 0; the rest is cleared by the caller).
template <bool EM = false>
__global__ void k_init_f2d(SolveArgs A, int ncells) {
  for (int cell = blockIdx.y; cell < ncells; cell += gridDim.y) {
    const CellDev c = A.cells[cell];
    const long long items = (long long)A.L * c.n * NP;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < items; i += (long long)gridDim.x * blockDim.x) {
      const int k = (int)(i % NP);
      const long long r = i / NP;
      const int y = (int)(r % c.n);
      const int l = (int)(r / c.n);
      const double* El = A.E + ((size_t)cell * A.L + l) * NP;
      double v = El[k];
      if (EM) {
        v = 2.0 * (2.0 * c.mu0 * El[k] + (k < 2 ? c.lam0 * (El[0] + El[1]) : 0.0));
        if (y == 0) {  // u_hat(0): component k of lane A at position 0, (re, im) in float2 slot k
          float2* ub = reinterpret_cast<float2*>(static_cast<float4*>(A.g) + (c.g_off + (size_t)l * (c.Hp / 2) * c.n * 6) / 2);
          ub[k] = make_float2((float)v, 0.f);
        }
      }
      static_cast<float4*>(A.eps[0])[tile_index(c, c.n, l, 0, y) + k] = make_float4((float)v, 0.f, 0.f, 0.f);
    }
  }
}

// ------------------------------------------------------------------ Green pass
// Eyre-Milton scheme: the positions of one thread, lane by lane through em_core (hom_em.cuh); the
// private state is u_hat of the current iterate, [position][6 complex] = (kx0 components 0..2, kx0+1
// components 0..2) as three float4, in place of g.  Returns the three compensated sums.
template <int N>
__device__ __forceinline__ void green_em(const SolveArgs& A, int kx0, bool hasB, const CellDev& c, const float* sx,
                                         const FastPlanDev& fp, float4* s, float4* ub, const double* Eld,
                                         Acc<float> (&acc)[3]) {
  CellConst<float> cc;
  cell_const(c, cc);
  const float nvT = (float)c.nv, inv_nv = cc.inv_nv, lam0 = cc.lam0, mu2_0 = cc.mu2;
  const float a0 = cc.lam0 / (cc.mu2 + 2.f * cc.lam0), inv_mu2_0 = 0.5f * cc.inv_mu0;
  const float X[2] = {__ldg(fp.xinat + kx0), hasB ? __ldg(fp.xinat + kx0 + 1) : 0.f};
  float* sf = reinterpret_cast<float*>(s);
  float2* u2 = reinterpret_cast<float2*>(ub);  // [position][lane A comps 0..2, lane B comps 0..2]
  // one (position, lane) per item: lane h reads and writes its own floats of the lane pairs
  for (int i = threadIdx.x; i < 2 * N; i += kT) {
    const int pos = i >> 1, h = i & 1;
    if (h && !hasB) continue;
    float2 th[NP], uh[NP], un[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      const float* T = sf + 4 * (pos * NP + k);  // (re A, re B, im A, im B)
      th[k] = make_float2(T[h], T[2 + h]);
      uh[k] = u2[6 * pos + 3 * h + k];
    }
    const float xi[2] = {X[h], sx[pos]};
    em_core<float, 2>(th, uh, un, xi, h == 0 && kx0 == 0 && pos == 0, false, h == 0 && kx0 == 0, nvT, inv_nv, lam0,
                      mu2_0, a0, inv_mu2_0, cc.inv_mu0, cc.ratio, Eld, acc[0], acc[1], acc[2]);
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      float* T = sf + 4 * (pos * NP + k);
      T[h] = un[k].x;
      T[2 + h] = un[k].y;
      u2[6 * pos + 3 * h + k] = un[k];
    }
  }
  if (!hasB)  // the missing lane B of the last pair stays zero
    for (int i = threadIdx.x; i < N * NP; i += kT) {
      sf[4 * i + 1] = 0.f;
      sf[4 * i + 3] = 0.f;
    }
}

// The finished tile (natural order after the inverse transform) -> the next eps buffer.
template <int N>
__device__ __forceinline__ void green_store(const SolveArgs& A, const float4* s, float4* out) {
#if HOM_GREEN_BULK
  fence_proxy_async();  // this thread's tile writes, visible to the bulk copy
  __syncthreads();
  if (threadIdx.x == 0) {
    bulk_store(out, s, (unsigned)(N * NP * sizeof(float4)));
    bulk_store_wait_read();  // the CTA keeps its shared memory until the copy has read it
  }
#else
  for (int f = threadIdx.x; f < N * NP; f += kT) out[f] = s[f];
#endif
  (void)A;
}

// tau (mixed domain) -> forward y-DFT -> Gamma0 and the residual on J (eq. 2) -> inverse y-DFT -> eps.
template <int N, bool EM = false>
__device__ __forceinline__ void green_body(const SolveArgs& A, int task, const TaskL& t, const CellDev& c,
                                           const FastPlanDev& fp, float4* s) {
  constexpr int H = (N + 1) / 2;
  const int cl = t.cell * A.L + t.load;
  if (!A.active[cl]) return;
  const int it = *A.it_dev;
  const int Hp = c.Hp, kx0 = t.kx0;
  const bool hasB = kx0 + 1 < H;
  // this task's tile (pair kx0 / 2 of its load): n rows x 3 components, contiguous
  const size_t tb = tile_index(c, N, t.load, kx0 / 2, 0);
  const float4* in = static_cast<const float4*>(A.tau) + tb;
  float4* out = static_cast<float4*>(A.eps[(it + 1) & 1]) + tb;
  const float2 z2 = make_float2(0.f, 0.f);
  // g of this column pair, [position][4 complex] = (kx0 d0, kx0 d1, kx0+1 d0, kx0+1 d1)
  float4* gb = static_cast<float4*>(A.g) +
               (c.g_off + ((size_t)t.load * (Hp / 2) + (size_t)(kx0 / 2)) * N * 4) / 2;
  // tile, twiddles and the wave numbers of the positions -> shared memory
#if HOM_GREEN_TW2
  float2* tws = reinterpret_cast<float2*>(s + N * NP);  // scalar twiddles: 3 CTAs per SM fit
  float* sx = reinterpret_cast<float*>(s + N * NP + (N + 1) / 2);
  for (int i = threadIdx.x; i < (N + 1) / 2; i += kT) cp16(tws + 2 * i, fp.tw2 + 2 * i);
#else
  float4* tws = s + N * NP;
  float* sx = reinterpret_cast<float*>(tws + N);
  for (int i = threadIdx.x; i < N; i += kT) cp16(tws + i, fp.tw4 + i);
#endif
#if HOM_GREEN_BULK
  // the tile (N NP float4, contiguous in HBM and in shared memory) by one bulk copy
  __shared__ __align__(8) unsigned long long tile_bar;
  fence_proxy_async();  // earlier generic writes to this shared memory are ordered before the copy's
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_init(&tile_bar, 1);
    bulk_load(s, in, (unsigned)(N * NP * sizeof(float4)), &tile_bar);
  }
#else
  for (int i = threadIdx.x; i < N * NP; i += kT) cp16(s + i, in + i);
#endif
  for (int i = threadIdx.x; i < (N + 3) / 4; i += kT) cp16(sx + 4 * i, fp.xipos + 4 * i);
  cp_commit();
  cp_wait_all();
#if HOM_GREEN_BULK
  __syncthreads();  // the barrier's initialisation is visible before anyone waits on it
  // bounded wait (a copy of 60 KB lands in microseconds); running out is recorded, never a hang
  if (!mbar_wait(&tile_bar, 0, 1 << 22) && A.dbg) atomicCAS(A.dbg, 0u, 0xFFFFFFFFu);
  __syncthreads();
  if (threadIdx.x == 0) mbar_inval(&tile_bar);
#endif
  __syncthreads();
#if HOM_GREEN_GPF
  // the private state of this column pair (contiguous: N positions x 2 or 3 float4) -> L2, so that
  // its reads after the transform hit L2
  if (threadIdx.x < 32) {
    const size_t per = EM ? 3 : 2;
    const char* gsrc = reinterpret_cast<const char*>(static_cast<const float4*>(A.g) +
                                                     (c.g_off + ((size_t)t.load * (Hp / 2) + (size_t)(kx0 / 2)) * N * 2 * per) / 2);
    const unsigned bytes = (unsigned)(N * per * sizeof(float4));
    constexpr unsigned kPiece = 4096;
    for (unsigned o = threadIdx.x * kPiece; o < bytes; o += 32 * kPiece) prefetch_l2(gsrc + o, min(kPiece, bytes - o));
  }
#endif
  fft_dif_p<NP, N, true>(s, tws);  // forward: bin ky at position perm(ky)

  if constexpr (EM) {
    float4* ub = static_cast<float4*>(A.g) + (c.g_off + ((size_t)t.load * (Hp / 2) + (size_t)(kx0 / 2)) * N * 6) / 2;
    Acc<float> acc[3];
    green_em<N>(A, kx0, hasB, c, sx, fp, s, ub, A.E + (size_t)cl * NP, acc);
    double tot[3];
    block_sum<float, 3, kT>(acc, tot);  // contains the barrier before the inverse transform
    if (threadIdx.x == 0) {
      A.partC[2 * (size_t)task] = tot[0];
      A.partC[2 * (size_t)task + 1] = tot[1];
      A.partE[task] = tot[2];
    }
    fft_dit_p<NP, N, false>(s, tws);  // inverse: natural order
    green_store<N>(A, s, out);
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
  const float2 X2 = mul2(X, X);
  const float2 wgt = make_float2(kx0 == 0 ? 1.f : 2.f, hasB ? 2.f : 0.f);
  const double* Eld = A.E + (size_t)cl * NP;
  float2 r2s = z2, r2c = z2, rns = z2, rnc = z2;  // Kahan sums (value, lost low part) per lane
  // g of every position of this thread, loaded at once
  constexpr int NPOS = (N + kT - 1) / kT;
  float4 gr[NPOS][2];
#pragma unroll
  for (int i = 0; i < NPOS; ++i) {
    const int pos = threadIdx.x + i * kT;
    if (pos < N) {
      gr[i][0] = gb[2 * pos];
      gr[i][1] = gb[2 * pos + 1];
    }
  }
#pragma unroll
  for (int i = 0; i < NPOS; ++i) {
    const int pos = threadIdx.x + i * kT;
    if (pos >= N) break;
    const float4 ga = gr[i][0], gbv = gr[i][1];
    const float2 Y = f2(sx[pos]);
    const P2 T0 = ldp(s[pos * NP]), T1 = ldp(s[pos * NP + 1]), T2 = ldp(s[pos * NP + 2]);
    const P2 G0{make_float2(ga.x, gbv.x), make_float2(ga.y, gbv.y)};
    const P2 G1{make_float2(ga.z, gbv.z), make_float2(ga.w, gbv.w)};
    // v = tau_hat . xi (tau_01 = T2 / sqrt 2)
    const P2 T01 = scale(rs2, T2);
    const P2 V0{fma2(Y, T01.re, mul2(X, T0.re)), fma2(Y, T01.im, mul2(X, T0.im))};
    const P2 V1{fma2(Y, T1.re, mul2(X, T01.re)), fma2(Y, T1.im, mul2(X, T01.im))};
    const float2 q2 = fma2(Y, Y, X2);
    const P2 XG{fma2(Y, G1.re, mul2(X, G0.re)), fma2(Y, G1.im, mul2(X, G0.im))};
    const P2 XV{fma2(Y, V1.re, mul2(X, V0.re)), fma2(Y, V1.im, mul2(X, V0.im))};
    // residual of the current iterate: r = tau_hat xi - K0 g, K0 g = mu0 q2 g + (lam0 + mu0) xi (xi . g)
    const float2 mq = mul2(mu0, q2);
    const float2 lx = mul2(lpm, X), ly = mul2(lpm, Y);
    const P2 R0{sub2(sub2(V0.re, mul2(mq, G0.re)), mul2(lx, XG.re)), sub2(sub2(V0.im, mul2(mq, G0.im)), mul2(lx, XG.im))};
    const P2 R1{sub2(sub2(V1.re, mul2(mq, G1.re)), mul2(ly, XG.re)), sub2(sub2(V1.im, mul2(mq, G1.im)), mul2(ly, XG.im))};
    float2 r2 = mul2(R0.re, R0.re);
    r2 = fma2(R0.im, R0.im, r2);
    r2 = fma2(R1.re, R1.re, r2);
    r2 = fma2(R1.im, R1.im, r2);
    const bool k0 = kx0 == 0 && pos == 0;  // k = 0: eps_hat(0) = E, g = 0, no residual
    const float2 iq = make_float2(k0 ? 0.f : __fdividef(1.f, q2.x), hasB ? __fdividef(1.f, q2.y) : 0.f);
    // g' = K0^-1 (tau_hat xi), eps_hat' = -sym(xi (x) g') / N_v
    const float2 imq = mul2(inv_mu0, iq);
    const float2 rq = mul2(ratio, iq);
    const float2 rx = mul2(rq, X), ry = mul2(rq, Y);
    const P2 W0{mul2(imq, sub2(V0.re, mul2(rx, XV.re))), mul2(imq, sub2(V0.im, mul2(rx, XV.im)))};
    const P2 W1{mul2(imq, sub2(V1.re, mul2(ry, XV.re))), mul2(imq, sub2(V1.im, mul2(ry, XV.im)))};
    const float2 nx = mul2(X, f2(-inv_nv)), ny = mul2(Y, f2(-inv_nv));
    const float2 ns = f2(-rs2 * inv_nv);
    P2 E0{mul2(nx, W0.re), mul2(nx, W0.im)};
    P2 E1{mul2(ny, W1.re), mul2(ny, W1.im)};
    P2 E2{mul2(ns, fma2(X, W1.re, mul2(Y, W0.re))), mul2(ns, fma2(X, W1.im, mul2(Y, W0.im)))};
    float4 gna = make_float4(W0.re.x, W0.im.x, W1.re.x, W1.im.x);
    const float4 gnb = make_float4(W0.re.y, W0.im.y, W1.re.y, W1.im.y);
    float2 wr = wgt;
    if (k0) {
      E0.re.x = (float)Eld[0]; E0.im.x = 0.f;
      E1.re.x = (float)Eld[1]; E1.im.x = 0.f;
      E2.re.x = (float)Eld[2]; E2.im.x = 0.f;
      gna = make_float4(0.f, 0.f, 0.f, 0.f);
      wr.x = 0.f;
    }
    s[pos * NP] = stp(E0);
    s[pos * NP + 1] = stp(E1);
    s[pos * NP + 2] = stp(E2);
    gb[2 * pos] = gna;
    gb[2 * pos + 1] = gnb;
    // Kahan accumulation of wgt * r2 and wgt * r2 / q2, lane by lane
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
    // combine the two lanes (each a compensated pair) into one compensated pair per sum
    vv[0].s = r2s.x;
    vv[0].c = r2c.x;
    vv[0].add(r2s.y);
    vv[0].add(-r2c.y);
    vv[1].s = rns.x;
    vv[1].c = rnc.x;
    vv[1].add(rns.y);
    vv[1].add(-rnc.y);
    double tot[2];
    block_sum<float, 2, kT>(vv, tot);  // contains the barrier before the inverse transform
    if (threadIdx.x == 0) {
      A.partC[2 * (size_t)task] = tot[0];
      A.partC[2 * (size_t)task + 1] = tot[1];
    }
  }
  fft_dit_p<NP, N, false>(s, tws);  // inverse: natural order
  green_store<N>(A, s, out);
  if (threadIdx.x == 0) {
    const int ntk = hasB ? 2 : 1;
    atomicAdd(A.bytes + HOM_K_GREEN,
              (unsigned long long)(2 * (size_t)N * ntk * NP * sizeof(float2) + 2 * (size_t)N * ntk * 2 * sizeof(float2)));
  }
}

// L2 prefetch of Green task `task`'s tau tile and g block (contiguous, in 4 KB pieces).
__device__ __forceinline__ void prefetch_green_task(const SolveArgs& A, int task) {
  const TaskL t = A.tC[task];
  if (!A.active[t.cell * A.L + t.load]) return;
  const CellDev c = A.cells[t.cell];
  const char* tau = reinterpret_cast<const char*>(static_cast<const float4*>(A.tau) + tile_index(c, c.n, t.load, t.kx0 / 2, 0));
  const char* g = reinterpret_cast<const char*>(static_cast<const float4*>(A.g) +
                                                (c.g_off + ((size_t)t.load * (c.Hp / 2) + (size_t)(t.kx0 / 2)) * c.n * 4) / 2);
  const unsigned bt = (unsigned)c.n * NP * sizeof(float4), bg = (unsigned)c.n * 2 * sizeof(float4);  // basic scheme's g
  constexpr unsigned kPiece = 4096;
  const unsigned nt = (bt + kPiece - 1) / kPiece, ng = (bg + kPiece - 1) / kPiece;
  for (unsigned i = threadIdx.x; i < nt + ng; i += kT) {
    const bool on_t = i < nt;
    const unsigned o = (on_t ? i : i - nt) * kPiece, b = on_t ? bt : bg;
    prefetch_l2((on_t ? tau : g) + o, min(kPiece, b - o));
  }
}

// One CTA per task; CTA b prefetches task b + ahead into L2 (see k_row_f2d).
template <bool EM = false>
__global__ void __launch_bounds__(kT, HOM_GREEN_TW2 ? 3 : 2) k_green_f2d(SolveArgs A, int ntasks, int ahead) {
  HOM_DBG_POISON();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float4* s = reinterpret_cast<float4*>(smem_raw);
  const int task = blockIdx.x;
  if (HOM_GREEN_PREFETCH && task + ahead < ntasks) prefetch_green_task(A, task + ahead);
  const TaskL t = A.tC[task];
  const CellDev c = A.cells[t.cell];
  // debug builds: an even kx pair start inside the half spectrum, a valid load
  if (!HOM_CHECK(A, t.kx0 >= 0 && (t.kx0 & 1) == 0 && t.kx0 < c.H && t.load >= 0 && t.load < A.L, (size_t)task))
    return;
  const FastPlanDev fp = A.fplans[c.fplan];
  switch (c.n) {
    case 45: green_body<45, EM>(A, task, t, c, fp, s); break;
    case 75: green_body<75, EM>(A, task, t, c, fp, s); break;
    case 135: green_body<135, EM>(A, task, t, c, fp, s); break;
    case 225: green_body<225, EM>(A, task, t, c, fp, s); break;
    case 405: green_body<405, EM>(A, task, t, c, fp, s); break;
    case 1215: green_body<1215, EM>(A, task, t, c, fp, s); break;
    default: break;
  }
}

// ------------------------------------------------------------------ labels in transform order
__global__ void k_permute_labels(SolveArgs A, int ncells) {
  const int ci = blockIdx.y;
  if (ci >= ncells) return;
  const CellDev c = A.cells[ci];
  if (c.fplan < 0) return;
  const FastPlanDev fp = A.fplans[c.fplan];
  const long long nv = c.nv;  // rows x n (rows are y in 2D, z n + y in 3D)
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (long long)gridDim.x * blockDim.x) {
    const long long y = i / c.n;
    const int pos = (int)(i - y * c.n);
    const uint32_t lab = A.label[c.vox_off + y * c.n + fp.iperm[pos]];
    const int nl = (c.n + 15) / 16 * 16;
    // local index of a pure voxel's phase in the cell's list (not found: the full-label path)
    uint32_t loc = kLabel8Mixed;
    if (!(lab & HOM_MIXED_BIT))
      for (int j = 0; j < c.nph; ++j)
        if ((uint32_t)A.cell_phases[c.ph_off + j] == lab) {
          loc = (uint32_t)j;
          break;
        }
    const_cast<uint8_t*>(A.label8)[c.lp_off + y * nl + pos] = (uint8_t)loc;
  }
}

// ------------------------------------------------------------------ host side
struct FastCacheEntry {
  int dev, n;
  FastPlanDev p;
  void* mem;
};
std::mutex g_fast_mu;
std::vector<FastCacheEntry> g_fast_cache;

std::vector<int> radices_of(int n) {
  switch (n) {
    case 45: return {Radix<45>::r0, Radix<45>::r1};
    case 75: return {Radix<75>::r0, Radix<75>::r1};
    case 135: return {Radix<135>::r0, Radix<135>::r1};
    case 225: return {Radix<225>::r0, Radix<225>::r1};
    case 405: return {Radix<405>::r0, Radix<405>::r1, Radix<405>::r2};
    case 1215: return {Radix<1215>::r0, Radix<1215>::r1, Radix<1215>::r2};
    case 27: return {Radix<27>::r0, Radix<27>::r1};
    case 81: return {Radix<81>::r0, Radix<81>::r1};
    case 243: return {Radix<243>::r0, Radix<243>::r1, Radix<243>::r2};
    default: return {};
  }
}

}  // namespace

bool fast2d_size(int n) {
  for (int k : kFastSizes)
    if (k == n) return true;
  return false;
}

int fast2d_plan_host(int n, std::vector<unsigned char>& h, FastPlanDev* out) {
  HostPlan hp;
  if (radices_of(n).empty() || !build_host_plan_radices(n, radices_of(n), hp))
    return set_error(HOM_ERR_UNSUPPORTED_SIZE, "no specialised plan for n = %d", n);
  auto up = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t b_tw = up((size_t)n * 16), b_ip = up((size_t)n * 2), b_xp = up((size_t)n * 4), b_xn = up((size_t)n * 4),
               b_t2 = up((size_t)n * 8 + 8);
  h.assign(b_tw + b_ip + b_xp + b_xn + b_t2, 0);
  // per-stage twiddle tables (stages with span L > 1): entry (q - 1) L + j = w^(j q n / (L R))
  float* tw = reinterpret_cast<float*>(h.data());
  {
    size_t e = 0;
    for (size_t st = 1; st < hp.radix.size(); ++st) {
      const int R = hp.radix[st], L = hp.span[st], TS = n / (L * R);
      for (int q = 1; q < R; ++q)
        for (int j = 0; j < L; ++j, ++e) {
          const int t = (j * q * TS) % n;
          tw[4 * e] = tw[4 * e + 1] = (float)hp.tw[2 * t];
          tw[4 * e + 2] = tw[4 * e + 3] = (float)hp.tw[2 * t + 1];
          float* t2 = reinterpret_cast<float*>(h.data() + b_tw + b_ip + b_xp + b_xn);
          t2[2 * e] = (float)hp.tw[2 * t];
          t2[2 * e + 1] = (float)hp.tw[2 * t + 1];
        }
    }
  }
  uint16_t* ip = reinterpret_cast<uint16_t*>(h.data() + b_tw);
  for (int k = 0; k < n; ++k) ip[hp.perm[k]] = (uint16_t)k;
  float* xp = reinterpret_cast<float*>(h.data() + b_tw + b_ip);
  float* xn = reinterpret_cast<float*>(h.data() + b_tw + b_ip + b_xp);
  for (int p = 0; p < n; ++p) xp[p] = (float)hp.xi[ip[p]];
  for (int k = 0; k < n; ++k) xn[k] = (float)hp.xi[k];
  // table pointers as byte offsets from the start of the tables (fast2d_plan_rebase adds the base)
  FastPlanDev p{};
  p.tw4 = reinterpret_cast<const float4*>(size_t(0));
  p.iperm = reinterpret_cast<const uint16_t*>(b_tw);
  p.xipos = reinterpret_cast<const float*>(b_tw + b_ip);
  p.xinat = reinterpret_cast<const float*>(b_tw + b_ip + b_xp);
  p.tw2 = reinterpret_cast<const float2*>(b_tw + b_ip + b_xp + b_xn);
  p.n = n;
  *out = p;
  return HOM_OK;
}

void fast2d_plan_rebase(FastPlanDev& p, const unsigned char* base) {
  auto at = [&](const void* off) { return base + reinterpret_cast<size_t>(off); };
  p.tw4 = reinterpret_cast<const float4*>(at(p.tw4));
  p.iperm = reinterpret_cast<const uint16_t*>(at(p.iperm));
  p.xipos = reinterpret_cast<const float*>(at(p.xipos));
  p.xinat = reinterpret_cast<const float*>(at(p.xinat));
  p.tw2 = reinterpret_cast<const float2*>(at(p.tw2));
}

int fast2d_plan(int n, FastPlanDev* out) {
  int dev = 0;
  HOM_CUDA_TRY(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_fast_mu);
  for (const auto& e : g_fast_cache)
    if (e.dev == dev && e.n == n) {
      *out = e.p;
      return HOM_OK;
    }
  std::vector<unsigned char> h;
  FastPlanDev p{};
  int rc = fast2d_plan_host(n, h, &p);
  if (rc != HOM_OK) return rc;
  void* mem = nullptr;
  HOM_CUDA_TRY(cudaMalloc(&mem, h.size()));
  HOM_CUDA_TRY(cudaMemcpy(mem, h.data(), h.size(), cudaMemcpyHostToDevice));
  fast2d_plan_rebase(p, static_cast<const unsigned char*>(mem));
  g_fast_cache.push_back({dev, n, p, mem});
  *out = p;
  return HOM_OK;
}

void fast2d_release() {
  std::lock_guard<std::mutex> lk(g_fast_mu);
  for (auto& e : g_fast_cache) {
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(e.dev);
    cudaFree(e.mem);
    cudaSetDevice(cur);
  }
  g_fast_cache.clear();
}

// row: tile | one-byte labels of 4 rows | twiddles | spare landing slots | per-phase update constants
// Green: tile | twiddles | wave numbers
size_t fast2d_smem_row(int nmax, int nphase_cell) {
  const size_t labels = (size_t)kFastRows * ((nmax + 15) / 16 * 16);
  const size_t tw = HOM_ROW_TW2 ? ((size_t)nmax + 1) / 2 * 16 : (size_t)nmax * sizeof(float4);
  return (size_t)nmax * NP * sizeof(float4) + labels + tw + (size_t)kRowSpare * sizeof(float4) +
         ((size_t)nphase_cell * 16 + 15) / 16 * 16;  // two float2 per phase (the second for the Eyre-Milton scheme)
}
size_t fast2d_smem_green(int nmax) {
  const size_t tw = HOM_GREEN_TW2 ? ((size_t)nmax + 1) / 2 * 16 : (size_t)nmax * sizeof(float4);
  return (size_t)nmax * NP * sizeof(float4) + tw + ((size_t)nmax + 3) / 4 * 16;
}

namespace {
template <typename K>
int opt_in(K kernel, size_t bytes) {
  if (bytes > 48 * 1024) HOM_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  return HOM_OK;
}
}  // namespace

int fast2d_row(const SolveArgs& A, unsigned ntasks, size_t smem, cudaStream_t st) {
  if (A.scheme == HOM_SCHEME_EYRE_MILTON) {
    int rc = opt_in(k_row_f2d<false, false, true>, smem);
    if (rc != HOM_OK) return rc;
    k_row_f2d<false, false, true><<<ntasks, kT, smem, st>>>(A, (int)ntasks,
                                                            resident_ctas(k_row_f2d<false, false, true>, kT, smem));
    return HOM_OK;
  }
  if (A.src) {  // adjoint solve: the constitutive step takes the source term
    int rc = opt_in(k_row_f2d<false, true>, smem);
    if (rc != HOM_OK) return rc;
    k_row_f2d<false, true><<<ntasks, kT, smem, st>>>(A, (int)ntasks, resident_ctas(k_row_f2d<false, true>, kT, smem));
    return HOM_OK;
  }
  int rc = opt_in(k_row_f2d<false, false>, smem);
  if (rc != HOM_OK) return rc;
  k_row_f2d<false, false><<<ntasks, kT, smem, st>>>(A, (int)ntasks, resident_ctas(k_row_f2d<false, false>, kT, smem));
  return HOM_OK;
}

int fast2d_out(const SolveArgs& A, unsigned ntasks, size_t smem, cudaStream_t st) {
  if (A.scheme == HOM_SCHEME_EYRE_MILTON) {
    int rc = opt_in(k_row_f2d<true, false, true>, smem);
    if (rc != HOM_OK) return rc;
    k_row_f2d<true, false, true><<<ntasks, kT, smem, st>>>(A, (int)ntasks,
                                                           resident_ctas(k_row_f2d<true, false, true>, kT, smem));
    return HOM_OK;
  }
  int rc = opt_in(k_row_f2d<true, false>, smem);
  if (rc != HOM_OK) return rc;
  k_row_f2d<true, false><<<ntasks, kT, smem, st>>>(A, (int)ntasks, resident_ctas(k_row_f2d<true, false>, kT, smem));
  return HOM_OK;
}

int fast2d_init(const SolveArgs& A, int ncells, cudaStream_t st) {
  dim3 grid(64, (unsigned)std::min(ncells, 65535));
  if (A.scheme == HOM_SCHEME_EYRE_MILTON) k_init_f2d<true><<<grid, 256, 0, st>>>(A, ncells);
  else k_init_f2d<false><<<grid, 256, 0, st>>>(A, ncells);
  return HOM_OK;
}

int fast2d_green(const SolveArgs& A, unsigned ntasks, size_t smem, cudaStream_t st) {
  if (A.scheme == HOM_SCHEME_EYRE_MILTON) {
    int rc = opt_in(k_green_f2d<true>, smem);
    if (rc != HOM_OK) return rc;
    k_green_f2d<true><<<ntasks, kT, smem, st>>>(A, (int)ntasks, resident_ctas(k_green_f2d<true>, kT, smem));
    return HOM_OK;
  }
  int rc = opt_in(k_green_f2d<false>, smem);
  if (rc != HOM_OK) return rc;
  k_green_f2d<false><<<ntasks, kT, smem, st>>>(A, (int)ntasks, resident_ctas(k_green_f2d<false>, kT, smem));
  return HOM_OK;
}

int fast2d_permute_labels(const SolveArgs& A, int ncells, long long max_nv, cudaStream_t st) {
  if (ncells > 65535) return set_error(HOM_ERR_UNSUPPORTED_SIZE, "too many cells for the label permutation");
  const unsigned gx = (unsigned)std::min<long long>((max_nv + 255) / 256, 1024);
  k_permute_labels<<<dim3(gx, (unsigned)ncells), 256, 0, st>>>(A, ncells);
  HOM_CUDA_TRY(cudaGetLastError());
  return HOM_OK;
}

}  // namespace hom

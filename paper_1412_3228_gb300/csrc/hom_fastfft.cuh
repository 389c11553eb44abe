// Shared core of the specialised FP32 passes (2D: hom_fast2d.cu, 3D: hom_fast3d.cu): packed FP32x2
// arithmetic on lane pairs, register DFTs, compile-time radix plans and the in-place mixed-radix
// DIT/DIF stages over a shared-memory tile of NP lane pairs per position (see hom_fast2d.cu for the
// lane-pair layout).  Included by one translation unit per dimension; everything here has
// internal linkage.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>

#include "hom_common.cuh"
#include "hom_fast2d.h"

namespace hom {
namespace {

#ifndef HOM_FAST_THREADS
#define HOM_FAST_THREADS 256
#endif
constexpr int kT = HOM_FAST_THREADS;  // threads per CTA (a build-time tunable)

// CTAs of `kernel` resident on the device at once (the prefetch distance of the passes), cached
// per kernel for the last (device, shared-memory size) asked.
template <typename K>
int resident_ctas(K kernel, int threads, size_t smem) {
  struct Last { const void* k = nullptr; int dev = -1; size_t smem = 0; int val = 0; };
  static thread_local Last last[4];
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  const void* kp = reinterpret_cast<const void*>(kernel);
  for (const Last& e : last)
    if (e.k == kp && e.dev == dev && e.smem == smem) return e.val;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    per_sm = 1;
  }
  static thread_local int next = 0;
  last[next] = Last{kp, dev, smem, std::max(sms, 1) * per_sm};
  const int v = last[next].val;
  next = (next + 1) & 3;
  return v;
}

// ------------------------------------------------------------------ packed FP32x2 arithmetic
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// a - b as b * (-1) + a: one rounding, the same result as a subtraction
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }

// 16-byte asynchronous global -> shared copies (completed by cp_wait_all + a barrier).
__device__ __forceinline__ void cp16(void* smem_dst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// 16-byte asynchronous copy that reads `bytes` (16 or 0) from global memory and zero-fills the rest.
__device__ __forceinline__ void cp16z(void* smem_dst, const void* gsrc, unsigned bytes) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(gsrc), "r"(bytes) : "memory");
}

// Bulk prefetch of `bytes` (a multiple of 16, 16-byte aligned) of global memory into L2; no
// completion to wait for.
__device__ __forceinline__ void prefetch_l2(const void* gsrc, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(gsrc), "r"(bytes) : "memory");
}

// ------------------------------------------------------------------ 1D bulk copies (TMA unit)
// Global -> shared completing on an mbarrier (transaction bytes), shared -> global in a bulk group.
// Both addresses 16-byte aligned, sizes multiples of 16.
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_inval(unsigned long long* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void bulk_load(void* sdst, const void* gsrc, unsigned bytes, unsigned long long* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(sdst)),
               "l"(gsrc), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
// Waits for phase `parity` of the barrier to complete, at most `budget` polls; false if it ran out.
// HOM_MBAR_SUSPEND_NS > 0 lets each poll suspend the thread up to that many nanoseconds.
#ifndef HOM_MBAR_SUSPEND_NS
#define HOM_MBAR_SUSPEND_NS 0
#endif
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, int budget) {
  for (int i = 0; i < budget; ++i) {
    unsigned done;
#if HOM_MBAR_SUSPEND_NS > 0
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity), "r"((unsigned)HOM_MBAR_SUSPEND_NS)
        : "memory");
#else
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
#endif
    if (done) return true;
  }
  return false;
}
// generic-proxy writes of this thread to shared memory, made visible to the bulk-copy unit
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void bulk_store(void* gdst, const void* ssrc, unsigned bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst), "r"(smem_u32(ssrc)),
               "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// waits until the bulk stores of this thread have read their shared-memory source
__device__ __forceinline__ void bulk_store_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }

// Landing slot of row r of kx pair p, component k, in a row pass (4 real rows = 2 complex lines).  A pair (kx = 2p, 2p + 1)
// produces the line positions 2p, 2p + 1, N - 2p - 1 and N - 2p, so its four rows land in those
// slots and the pair is expanded in place without touching another pair's data.  Pair 0 (kx = 0
// maps to itself) and, when the half spectrum has an odd length H, the last pair (kx = H is
// absent, so its positions collide) land in a spare area instead; the slots they produce (0, 1,
// N - 1, and H - 1, H) are no other pair's landing slots.
// (NC lane pairs per position, SP float4 between positions in shared memory; the spare area holds
// 2 NC kFastRows float4.)
template <int N, int NC, int SP>
__device__ __forceinline__ float4* row_slot_p(float4* s, float4* spare, int p, int k, int r) {
  constexpr int H = (N + 1) / 2, P = (H + 1) / 2;
  if (p == 0) return spare + k * kFastRows + r;
  if ((H & 1) && p == P - 1) return spare + (NC + k) * kFastRows + r;
  const int pos = r < 2 ? 2 * p + r : N - 2 * p - (3 - r);  // 2p, 2p + 1, N - 2p - 1, N - 2p
  return s + pos * SP + k;
}

// Two complex numbers, one per line: re = (re_A, re_B), im = (im_A, im_B).
struct P2 {
  float2 re, im;
};
__device__ __forceinline__ P2 ldp(const float4& v) { return P2{make_float2(v.x, v.y), make_float2(v.z, v.w)}; }
__device__ __forceinline__ float4 stp(const P2& p) { return make_float4(p.re.x, p.re.y, p.im.x, p.im.y); }
__device__ __forceinline__ P2 operator+(P2 a, P2 b) { return P2{add2(a.re, b.re), add2(a.im, b.im)}; }
__device__ __forceinline__ P2 operator-(P2 a, P2 b) { return P2{sub2(a.re, b.re), sub2(a.im, b.im)}; }
__device__ __forceinline__ P2 scale(float s, P2 a) { return P2{mul2(f2(s), a.re), mul2(f2(s), a.im)}; }
// a * w (FWD) or a * conj(w) with w4 = (wr, wr, wi, wi)
template <bool FWD>
__device__ __forceinline__ P2 twmul(P2 a, float4 w4) {
  const float2 wr = make_float2(w4.x, w4.y), wi = make_float2(w4.z, w4.w);
  if (FWD) return P2{sub2(mul2(a.re, wr), mul2(a.im, wi)), fma2(a.re, wi, mul2(a.im, wr))};
  return P2{fma2(a.im, wi, mul2(a.re, wr)), sub2(mul2(a.im, wr), mul2(a.re, wi))};
}

// a * w (FWD) or a * conj(w) with a scalar twiddle w = (wr, wi), broadcast to both lanes
template <bool FWD>
__device__ __forceinline__ P2 twmul(P2 a, float2 w) {
  return twmul<FWD>(a, make_float4(w.x, w.x, w.y, w.y));
}

// ------------------------------------------------------------------ butterfly constants
// Every constant the register DFTs multiply by, duplicated into a lane pair, in constant memory:
// the packed instructions can take such an operand without a register copy.
#define HOM_TWP(R, m)                                                                              \
  {(float)tw_cos(R, m), (float)tw_cos(R, m)}, {(float)tw_sin(R, m), (float)tw_sin(R, m)},          \
      {(float)-tw_sin(R, m), (float)-tw_sin(R, m)}
constexpr float kH3 = 0.866025403784438646763723170753f;  // sin(2 pi / 3)
constexpr float kC51 = 0.309016994374947424102293417183f, kC52 = -0.809016994374947424102293417183f;
constexpr float kS51 = 0.951056516295153572116439333379f, kS52 = 0.587785252292473129168705954639f;
enum { KMH = 0, KH3, KNH3, KC51, KC52, KS51, KS52, KNS51, KNS52, KTW9 };
constexpr int kTw15 = KTW9 + 27;
__constant__ float2 kP[kTw15 + 45] = {
    {-0.5f, -0.5f}, {kH3, kH3}, {-kH3, -kH3}, {kC51, kC51}, {kC52, kC52}, {kS51, kS51}, {kS52, kS52}, {-kS51, -kS51},
    {-kS52, -kS52},
    HOM_TWP(9, 0), HOM_TWP(9, 1), HOM_TWP(9, 2), HOM_TWP(9, 3), HOM_TWP(9, 4), HOM_TWP(9, 5), HOM_TWP(9, 6),
    HOM_TWP(9, 7), HOM_TWP(9, 8),
    HOM_TWP(15, 0), HOM_TWP(15, 1), HOM_TWP(15, 2), HOM_TWP(15, 3), HOM_TWP(15, 4), HOM_TWP(15, 5), HOM_TWP(15, 6),
    HOM_TWP(15, 7), HOM_TWP(15, 8), HOM_TWP(15, 9), HOM_TWP(15, 10), HOM_TWP(15, 11), HOM_TWP(15, 12),
    HOM_TWP(15, 13), HOM_TWP(15, 14)};
#undef HOM_TWP
template <int R> __device__ __forceinline__ constexpr int tw_base() { return R == 9 ? KTW9 : kTw15; }

// ------------------------------------------------------------------ register DFTs on lane pairs
// Forward transforms use w = exp(-2 pi i / r), inverse ones conj(w); no scaling.  Composite sizes
// leave X[k] in v[out_pos<R>(k)] (hom_common.cuh).
template <bool FWD>
__device__ __forceinline__ void dft3p(P2* v) {
  const P2 s = v[1] + v[2];
  const P2 d = v[1] - v[2];
  const P2 m{fma2(s.re, kP[KMH], v[0].re), fma2(s.im, kP[KMH], v[0].im)};
  v[0] = v[0] + s;
  // v1 = m - i hf d, v2 = m + i hf d with hf = +-sin(2 pi / 3)
  const float2 hp = kP[FWD ? KH3 : KNH3], hn = kP[FWD ? KNH3 : KH3];
  v[1] = P2{fma2(d.im, hp, m.re), fma2(d.re, hn, m.im)};
  v[2] = P2{fma2(d.im, hn, m.re), fma2(d.re, hp, m.im)};
}

template <bool FWD>
__device__ __forceinline__ void dft5p(P2* v) {
  const P2 a1 = v[1] + v[4], b1 = v[1] - v[4];
  const P2 a2 = v[2] + v[3], b2 = v[2] - v[3];
  const float2 c1 = kP[KC51], c2 = kP[KC52];
  const P2 r1{fma2(a2.re, c2, fma2(a1.re, c1, v[0].re)), fma2(a2.im, c2, fma2(a1.im, c1, v[0].im))};
  const P2 r2{fma2(a2.re, c1, fma2(a1.re, c2, v[0].re)), fma2(a2.im, c1, fma2(a1.im, c2, v[0].im))};
  // t1 = +-s1, t2 = +-s2: i1 = t1 b1 + t2 b2, i2 = t2 b1 - t1 b2
  const float2 t1 = kP[FWD ? KS51 : KNS51], t2 = kP[FWD ? KS52 : KNS52], nt1 = kP[FWD ? KNS51 : KS51];
  const P2 i1{fma2(b2.re, t2, mul2(b1.re, t1)), fma2(b2.im, t2, mul2(b1.im, t1))};
  const P2 i2{fma2(b2.re, nt1, mul2(b1.re, t2)), fma2(b2.im, nt1, mul2(b1.im, t2))};
  v[0] = v[0] + a1 + a2;
  // X1 = r1 - i i1, X4 = r1 + i i1, X2 = r2 - i i2, X3 = r2 + i i2
  v[1] = P2{add2(r1.re, i1.im), sub2(r1.im, i1.re)};
  v[4] = P2{sub2(r1.re, i1.im), add2(r1.im, i1.re)};
  v[2] = P2{add2(r2.re, i2.im), sub2(r2.im, i2.re)};
  v[3] = P2{sub2(r2.re, i2.im), add2(r2.im, i2.re)};
}

template <int R, bool FWD> __device__ __forceinline__ void dftp(P2* v);

// R = A * B inside the registers: X[ka + A kb] = sum_nb w_B^(nb kb) [w_R^(nb ka) sum_na x[B na + nb] w_A^(na ka)]
template <int A, int B, bool FWD>
__device__ __forceinline__ void dft_compositep(P2* v) {
  constexpr int R = A * B;
#pragma unroll
  for (int nb = 0; nb < B; ++nb) {
    P2 t[A];
#pragma unroll
    for (int na = 0; na < A; ++na) t[na] = v[B * na + nb];
    dftp<A, FWD>(t);
#pragma unroll
    for (int ka = 0; ka < A; ++ka) {
      const P2 x = t[out_pos<A>(ka)];
      const int m = (nb * ka) % R;
      if (m == 0) {
        v[B * ka + nb] = x;
      } else {
        // x (cos + i sn), sn = -+sin(2 pi m / R)
        const int b = tw_base<R>() + 3 * m;
        const float2 c = kP[b], sp = kP[b + 1], sm = kP[b + 2];
        const float2 sn = FWD ? sm : sp, nsn = FWD ? sp : sm;
        v[B * ka + nb] = P2{fma2(x.im, nsn, mul2(x.re, c)), fma2(x.im, c, mul2(x.re, sn))};
      }
    }
  }
#pragma unroll
  for (int ka = 0; ka < A; ++ka) dftp<B, FWD>(v + B * ka);
}

template <int R, bool FWD>
__device__ __forceinline__ void dftp(P2* v) {
  if constexpr (R == 3) dft3p<FWD>(v);
  else if constexpr (R == 5) dft5p<FWD>(v);
  else dft_compositep<split_a<R>(), R / split_a<R>(), FWD>(v);
}

// ------------------------------------------------------------------ compile-time plans
// Radices in DIT order; registers bound the radix at 15 (15 lane pairs = 60 floats).
template <int N> struct Radix;
template <> struct Radix<45> { static constexpr int m = 2, r0 = 5, r1 = 9, r2 = 1; };
template <> struct Radix<75> { static constexpr int m = 2, r0 = 5, r1 = 15, r2 = 1; };
template <> struct Radix<135> { static constexpr int m = 2, r0 = 15, r1 = 9, r2 = 1; };
template <> struct Radix<225> { static constexpr int m = 2, r0 = 15, r1 = 15, r2 = 1; };
template <> struct Radix<405> { static constexpr int m = 3, r0 = 5, r1 = 9, r2 = 9; };
template <> struct Radix<1215> { static constexpr int m = 3, r0 = 15, r1 = 9, r2 = 9; };
template <> struct Radix<27> { static constexpr int m = 2, r0 = 3, r1 = 9, r2 = 1; };
template <> struct Radix<81> { static constexpr int m = 2, r0 = 9, r1 = 9, r2 = 1; };
template <> struct Radix<243> { static constexpr int m = 3, r0 = 3, r1 = 9, r2 = 9; };

// Radix-9 stages with HOM_TW_POW: of the eight twiddles w^q (q = 1..8) of a butterfly only w and
// w^4 are read from the table; the others are products of at most three of them (w^2 = w w,
// w^3 = w^2 w, w^5 = w^4 w, w^6 = w^4 w^2, w^7 = w^4 w^3, w^8 = w^4 w^4), so each carries at most three
// extra roundings, in exchange for six fewer shared-memory reads per butterfly (HOM_TW_POW = 2:
// seven fewer, w^4 = w^2 w^2).
#ifndef HOM_TW_POW
#define HOM_TW_POW 1
#endif
__device__ __forceinline__ float2 cmul1(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 tw_scalar(const float4& t) { return make_float2(t.x, t.z); }
__device__ __forceinline__ float2 tw_scalar(const float2& t) { return t; }
template <typename TW>
__device__ __forceinline__ void tw_pow9(const TW* tw, int L, int j, float2 (&w)[9]) {
  w[1] = tw_scalar(tw[j]);
  w[2] = cmul1(w[1], w[1]);
  // HOM_TW_POW = 2 reads w alone and squares w^2 into w^4 (at most three roundings still)
  w[4] = HOM_TW_POW == 2 ? cmul1(w[2], w[2]) : tw_scalar(tw[3 * L + j]);
  w[3] = cmul1(w[2], w[1]);
  w[5] = cmul1(w[4], w[1]);
  w[6] = cmul1(w[4], w[2]);
  w[7] = cmul1(w[4], w[3]);
  w[8] = cmul1(w[4], w[4]);
}

// One stage over the NP pairs of every position; thread t takes the butterflies t, t + kT, ...
// (pair-major, so neighbouring threads take neighbouring butterflies of one pair).
// Twiddles of a stage with span L > 1 come from its own table, tw[(q - 1) L + j] = w^(j q n / (L R))
// (q = 1..R-1, j < L): neighbouring threads read neighbouring entries.
template <int NP, int N, int R, int L, bool FWD, bool DIT, typename TW, int SP = NP, int NT = kT>
__device__ __forceinline__ void stage_p(float4* s, const TW* tw) {
  constexpr int NB = N / R, B = L * R;
  for (int t = threadIdx.x; t < NB * NP; t += NT) {
    const int cc = t / NB;
    const int b = t - cc * NB;
    const int blk = b / L;
    const int j = b - blk * L;
    float4* base = s + (blk * B + j) * SP + cc;
    P2 v[R];
    constexpr bool kPow = HOM_TW_POW && R == 9 && L > 1;
    float2 wp[9];
    if constexpr (kPow) tw_pow9(tw, L, j, wp);
    if (DIT) {
      v[0] = ldp(base[0]);
#pragma unroll
      for (int q = 1; q < R; ++q) {
        P2 x = ldp(base[q * L * SP]);
        if constexpr (kPow) x = twmul<FWD>(x, wp[q]);
        else if (L > 1) x = twmul<FWD>(x, tw[(q - 1) * L + j]);
        v[q] = x;
      }
      dftp<R, FWD>(v);
#pragma unroll
      for (int p = 0; p < R; ++p) base[p * L * SP] = stp(v[out_pos<R>(p)]);
    } else {
#pragma unroll
      for (int q = 0; q < R; ++q) v[q] = ldp(base[q * L * SP]);
      dftp<R, FWD>(v);
      base[0] = stp(v[0]);
#pragma unroll
      for (int p = 1; p < R; ++p) {
        P2 x = v[out_pos<R>(p)];
        if constexpr (kPow) x = twmul<FWD>(x, wp[p]);
        else if (L > 1) x = twmul<FWD>(x, tw[(p - 1) * L + j]);
        base[p * L * SP] = stp(x);
      }
    }
  }
}

// Stage tables are stored back to back: stage 1 (span r0) first, then stage 2 (span r0 r1).
template <int NP, int N, bool FWD, typename TW, int SP = NP, int NT = kT>
__device__ __forceinline__ void fft_dit_p(float4* s, const TW* tw) {
  using P = Radix<N>;
  constexpr int off2 = P::r0 * (P::r1 - 1);
  stage_p<NP, N, P::r0, 1, FWD, true, TW, SP, NT>(s, tw);
  __syncthreads();
  if constexpr (P::m > 1) {
    stage_p<NP, N, P::r1, P::r0, FWD, true, TW, SP, NT>(s, tw);
    __syncthreads();
  }
  if constexpr (P::m > 2) {
    stage_p<NP, N, P::r2, P::r0 * P::r1, FWD, true, TW, SP, NT>(s, tw + off2);
    __syncthreads();
  }
}

template <int NP, int N, bool FWD, typename TW, int SP = NP, int NT = kT>
__device__ __forceinline__ void fft_dif_p(float4* s, const TW* tw) {
  using P = Radix<N>;
  constexpr int off2 = P::r0 * (P::r1 - 1);
  if constexpr (P::m > 2) {
    stage_p<NP, N, P::r2, P::r0 * P::r1, FWD, false, TW, SP, NT>(s, tw + off2);
    __syncthreads();
  }
  if constexpr (P::m > 1) {
    stage_p<NP, N, P::r1, P::r0, FWD, false, TW, SP, NT>(s, tw);
    __syncthreads();
  }
  stage_p<NP, N, P::r0, 1, FWD, false, TW, SP, NT>(s, tw);
  __syncthreads();
}

}  // namespace
}  // namespace hom

// lfm_solve.cuh -- shared by the single-case kernels (lfm_step.cu) and the batched kernel
// (lfm_batch.cu).
//
// Device code of one implicit-Euler time step of laplacianFoam
// (arXiv 2507.18268, Eq. (1) and the listing "laplacianFoam application": per step one
// solve of fvm::ddt(T) - fvm::laplacian(DT, T)).
//
// A team of CTAs runs the steps of one case. Each CTA owns a contiguous range of cells and, in
// every phase, computes whole matrix rows by gathering over the face-to-cell slots (the
// paper's atomic-free rewrite of the face loop, listing "First cycle gradient in
// parallel"): no atomics touch data and every reduction has a fixed order. A thread takes
// two cells per loop trip and issues all their loads before using any, so that each thread
// keeps a dozen independent memory requests in flight.
//
// The face coefficients -g, g = DT |Sf| deltaCoeff, depend on the mesh and DT only: the
// set-up kernel (coef_kernel, lfm_step.cu) stores them at both of each face's slots when
// those change; the step kernel assembles faces itself only for matrix read-back.
//
// FP64 step (phases separated by team barriers):
//   A1 sum             sum x for xRef
//   A2+I rows          diag, source, rD = 1/diag, row sum; from the same loaded row
//                      A x, r = b - A x, normFactor, sum|r|, w = rD r, rho; p = w (first
//                      search direction). The source is needed by no later phase of an
//                      FP64 step and is stored only for read-back.
//   loop (diagonal-preconditioned CG, convergence on sum|r| / normFactor):
//   P  p = w + beta p  (skipped on the first iteration)
//   M  q = A p, sigma = p.q                   -> alpha = rho / sigma
//   U  x += alpha p, r -= alpha q, w = rD r, sum|r|, rho' = w.r -> beta = rho'/rho
//
// General (non-orthogonal) meshes (section "Code Porting": the gradient passes): A1 also
// evaluates the Gauss linear gradient of T per cell, and A2 adds to each row's source the
// explicit correction of the corrected laplacian (the face fluxes DT |Sf| k . G_f summed
// over the cell's faces), both through operator weights built from the geometry when it,
// the patches or DT change. With n_corr > 0 every step runs 1 + n_corr assemble-and-solve
// passes, the ddt source taken from T at the start of the step (x_old).
//
// Mixed step (defect correction, FP64 field x; on orthogonal meshes the df64 variant in
// lfm_solve_df.cuh runs instead): the matrix is assembled in FP64 with FP32 copies of the
// diagonal and 1/diag (the FP32 off-diagonals are set-up data); each sweep computes the FP64
// true residual r = b - A x (the first one in the assembly's row pass), solves A dx = r by
// the same CG recurrence on FP32 vectors with FP32 row sums, and adds dx to x in FP64. Dot
// products, sum|r|, normFactor and every convergence test are FP64-accurate: FP64 for the
// FP64 quantities; for FP32 terms, exact products summed as unevaluated FP32 pairs per
// thread and FP64 across threads (see Acc2f).
#pragma once

#include <cuda_runtime.h>

#include "lfm_device.cuh"
#include "lfm_internal.h"

namespace lfm {
namespace {

constexpr double kSmall = 1e-20;    // added to normFactor
constexpr double kVSmall = 1e-300;  // singularity threshold on |p.Ap| / normFactor
constexpr double kInnerRel = 1e-6;  // mixed: inner solve stops at this fraction of the sweep's start residual

__device__ __forceinline__ bool converged(double res, double init_res, double tol, double rel_tol) {
  return res < tol || (rel_tol > 0.0 && res < rel_tol * init_res);
}

// Contiguous cell range [c0, c1) of this CTA.
__device__ __forceinline__ void cta_range(int N, int size, int rank, int& c0, int& c1) {
  int chunk = (N + size - 1) / size;
  chunk = (chunk + 31) & ~31;
  long long a = (long long)rank * chunk;
  c0 = (int)(a < N ? a : N);
  long long b = a + chunk;
  c1 = (int)(b < N ? b : N);
}

// Slot count: the compile-time width when the kernel is specialised, else the case's.
template <int W>
__device__ __forceinline__ int nslots(const CaseDev& cs) {
  return W > 0 ? W : cs.W;
}

// ---- FP64-accurate accumulation of FP32 terms without FP64 instructions -----------------
// A running sum kept as an unevaluated pair hi + lo of FP32 numbers: each product of two
// FP32 values is split exactly into p + e (e = fma(a, b, -p)), p enters hi through Knuth's
// TwoSum (whose rounding error is exact), and the error terms collect in lo. Over the tens
// of terms one thread adds per pass, hi + lo carries ~2^-44 relative error; each thread
// converts it to FP64 once, and the block and team reductions run in FP64. (The FP64 pipe
// is the scarce unit on GB300: converting every term would cost two FP64 issues each.)
struct Acc2f {
  float hi = 0.0f, lo = 0.0f;
  __device__ __forceinline__ void add(float v) {
    const float s = __fadd_rn(hi, v);
    const float bp = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(v, bp));
    hi = s;
    lo = __fadd_rn(lo, e);
  }
  __device__ __forceinline__ void add_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    const float e = __fmaf_rn(a, b, -p);
    add(p);
    lo = __fadd_rn(lo, e);
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// ---- assembly of fvm::ddt(T) - fvm::laplacian(DT, T) ----------------------------------
// Face part (per face, in face order): g = (DT |Sf|) deltaCoeff, computed once per face and
// stored as -g at the face's slot in its owner's row and in its neighbour's row. It depends
// on the mesh and DT only, so the set-up kernel (coef_kernel) forms it when those change
// (the a0 step: precomputed face conductances); the step kernel repeats it only for matrix
// read-back, where the face-indexed LDU copy is written too.
template <bool kMixed>
__device__ __forceinline__ void assemble_face(const CaseDev& cs, int f, bool write_upper) {
  const uint2 at0 = __ldg(reinterpret_cast<const uint2*>(cs.face_slots) + f);
  const uint2 at = make_uint2(LFM_IDX(at0.x, cs.W * cs.N, 0, kChkFaceSlot), LFM_IDX(at0.y, cs.W * cs.N, 0, kChkFaceSlot));
  const double DTf = cs.DT_is_uniform ? cs.DT_uniform : __ldg(cs.DT + f);
  const double g = __dmul_rn(__dmul_rn(DTf, __ldg(cs.magSf + f)), __ldg(cs.delta + f));
  cs.slot_coef[at.x] = -g;
  cs.slot_coef[at.y] = -g;
  if (kMixed) {
    cs.slot_coef32[at.x] = (float)(-g);
    cs.slot_coef32[at.y] = (float)(-g);
  }
  if (write_upper) cs.upper[f] = -g;  // the face-indexed LDU copy, for read-back only
}

// Pass 2 (per cell): the row's diagonal summed in slot order, i.e. ascending face order
// (neighbour-side faces have smaller owners, so they precede the cell's own faces in
// upper-triangular order), then the boundary faces, then V/dt, every product and sum rounded
// separately (no FMA); the source; the row sum of A (the off-diagonals cancel the face
// conductances in the diagonal exactly in real arithmetic, leaving V/dt plus the boundary
// conductance). The row's A x is formed from the same loaded coefficients (the off-diagonal
// products fused in slot order, then diag * x_c), so the initial residual needs no second
// pass over the matrix.
struct Row {
  double d, s, sa, ax, xc;
};

// Clears the sign of a zero (0.0 + v would, at the cost of an FP64 add).
__device__ __forceinline__ double plus_zero(double v) {
  const long long bits = __double_as_longlong(v);
  return (bits << 1) == 0 ? 0.0 : v;
}

// xo: T of the cell at the start of the step (the ddt source).
__device__ __forceinline__ void row_boundary(const CaseDev& cs, int c, double xo, Row& o) {
  const int b0 = __ldg(cs.b_start + c), b1 = __ldg(cs.b_start + c + 1);
  const double vdt = cs.vdt[c];  // V/dt, formed once per (mesh, dt): the same IEEE quotient
  const double sv = __dmul_rn(vdt, xo);
  if (b0 == b1) {  // no boundary face: the sums below start from zero
    o.d = __dadd_rn(o.d, vdt);
    o.s = plus_zero(sv);
    o.sa = vdt;
    return;
  }
  double s = 0.0, gsum = 0.0;  // source, boundary conductance of the row
  for (int k = b0; k < b1; ++k) {
    const int bf = LFM_IDX(__ldg(cs.b_face + k), cs.NB, 0, kChkBFace);
    if (__ldg(cs.btype + bf) == LFM_FIXED_VALUE) {
      const double gb = __dmul_rn(__dmul_rn(__ldg(cs.bDT + bf), __ldg(cs.bmagSf + bf)), __ldg(cs.bdelta + bf));
      o.d = __dadd_rn(o.d, gb);
      s = __dadd_rn(s, __dmul_rn(gb, __ldg(cs.bval + bf)));
      gsum = __dadd_rn(gsum, gb);
    }
  }
  o.d = __dadd_rn(o.d, vdt);
  o.s = __dadd_rn(s, sv);
  o.sa = gsum + vdt;
}

// ---- general geometry: Gauss gradient and the explicit non-orthogonal correction ---------
// Gauss linear gradient of x at cell c through the operator weights (gD, gH, gE; see
// CaseDev): one fused multiply-add per slot and component.
template <int W>
__device__ __forceinline__ void op_grad(const CaseDev& cs, int c, const double* __restrict__ x, double* g) {
  const size_t N = (size_t)cs.N;
  const int ns = W > 0 ? W : cs.W;
  const size_t WN = (size_t)ns * N;
  const double xc = x[c];
  double g0 = fma(__ldg(cs.gD + c), xc, __ldg(cs.gH + c));
  double g1 = fma(__ldg(cs.gD + N + c), xc, __ldg(cs.gH + N + c));
  double g2 = fma(__ldg(cs.gD + 2 * N + c), xc, __ldg(cs.gH + 2 * N + c));
#pragma unroll
  for (int k = 0; k < (W > 0 ? W : kMaxSlots); ++k) {
    if (W == 0 && k >= ns) break;
    const size_t at = (size_t)k * N + c;
    const double xo = x[LFM_IDX(__ldg(cs.slot_other + at), cs.N, c, kChkSlotCell)];
    g0 = fma(__ldg(cs.gE + at), xo, g0);
    g1 = fma(__ldg(cs.gE + WN + at), xo, g1);
    g2 = fma(__ldg(cs.gE + 2 * WN + at), xo, g2);
  }
  g[0] = g0;
  g[1] = g1;
  g[2] = g2;
}

// Explicit correction source of row c: the sum over the cell's faces of the correction flux
// (+ where it owns the face, - where it is the neighbour), through the weights cK, cL.
template <int W>
__device__ __forceinline__ double op_corr_source(const CaseDev& cs, int c) {
  const size_t N = (size_t)cs.N;
  const int ns = W > 0 ? W : cs.W;
  const size_t WN = (size_t)ns * N;
  const double* G = cs.grad;
  double v = __ldg(cs.cK + c) * G[c];
  v = fma(__ldg(cs.cK + N + c), G[N + c], v);
  v = fma(__ldg(cs.cK + 2 * N + c), G[2 * N + c], v);
#pragma unroll
  for (int k = 0; k < (W > 0 ? W : kMaxSlots); ++k) {
    if (W == 0 && k >= ns) break;
    const size_t at = (size_t)k * N + c;
    const int o = LFM_IDX(__ldg(cs.slot_other + at), cs.N, c, kChkSlotCell);
    v = fma(__ldg(cs.cL + at), G[o], v);
    v = fma(__ldg(cs.cL + WN + at), G[N + o], v);
    v = fma(__ldg(cs.cL + 2 * WN + at), G[2 * N + o], v);
  }
  return v;
}

// kCorr: the step has non-orthogonal corrector passes, general geometry or a volumetric
// source: the ddt source comes from x_old (with correctors), the source S_T = Su + Sp T
// enters (V Su to the source, -V Sp to the diagonal), and the explicit correction of the
// row's faces is added to the source.
template <int W, bool kCorr = false>
__device__ __forceinline__ Row assemble_row(const CaseDev& cs, int c, const double* __restrict__ x) {
  const size_t N = (size_t)cs.N;
  Row o;
  o.xc = x[c];
  o.d = 0.0;
  double off = 0.0;  // sum of the off-diagonal products, slot order
  if constexpr (W > 0) {
    int oc[W];
    double u[W];
#pragma unroll
    for (int k = 0; k < W; ++k) {
      oc[k] = LFM_IDX(__ldg(cs.slot_other + (size_t)k * N + c), cs.N, c, kChkSlotCell);
      u[k] = cs.slot_coef[(size_t)k * N + c];
    }
    // 0 + g_0 = g_0 exactly; the sign of a zero cannot reach d, which ends above V/dt > 0
    o.d = -u[0];
#pragma unroll
    for (int k = 1; k < W; ++k) o.d = __dadd_rn(o.d, -u[k]);  // padding slots hold 0
#pragma unroll
    for (int k = 0; k < W; ++k) off = fma(u[k], x[oc[k]], off);
  } else {
    const int ns = cs.W;
    for (int k = 0; k < ns; ++k) {
      const size_t at = (size_t)k * N + c;
      const double u = cs.slot_coef[at];
      o.d = __dadd_rn(o.d, -u);
      off = fma(u, x[LFM_IDX(__ldg(cs.slot_other + at), cs.N, c, kChkSlotCell)], off);
    }
  }
  row_boundary(cs, c, kCorr && cs.n_corr > 0 ? cs.x_old[c] : o.xc, o);
  if (kCorr && cs.vSp) {  // implicit part of the source S_T = Su + Sp T
    const double v = cs.vSp[c];
    o.d = __dsub_rn(o.d, v);
    o.sa = o.sa - v;
  }
  if (kCorr && cs.vSu) o.s = __dadd_rn(o.s, cs.vSu[c]);
  if (kCorr && cs.Sf) o.s = __dadd_rn(o.s, op_corr_source<W>(cs, c));
  o.ax = fma(o.d, o.xc, off);
  return o;
}

// Writes the assembled row (diag, source, 1/diag and the FP32 copies). Returns 1/diag.
template <bool kMixed>
__device__ __forceinline__ double store_row(const CaseDev& cs, int c, const Row& o, bool keep_src) {
  const double rd = __drcp_rn(o.d);  // IEEE round-to-nearest reciprocal, as 1.0 / d
  cs.diag[c] = o.d;
  cs.rD[c] = rd;
  if (keep_src) cs.src[c] = o.s;
  if (kMixed) {
    cs.diag32[c] = (float)o.d;
    cs.rD32[c] = (float)rd;
  }
  return rd;
}

// The per-step passes (faces, rows + initial residual, true residual) are compiled as
// functions of their own (__noinline__, taking an addressable copy of the case descriptor):
// their register demand then does not shape the allocation of the iteration passes.

// First phase of an assembly: this thread's sum of T over the cells [c0, c1) (for xRef).
// The face coefficients are set-up data (written by the set-up kernel when the mesh or DT
// change); with `faces` (matrix read-back) the faces [f0, f1) of this CTA are assembled here
// as well, the face-indexed LDU copy included.
// save_old: also keep T as the step's starting field (x_old) for the corrector passes.
template <int B, bool kMixed>
__device__ __noinline__ double pass_faces(const CaseDev& cs, int f0, int f1, int c0, int c1, bool faces,
                                          bool save_old) {
  if (faces)
    for (int f = f0 + (int)threadIdx.x; f < f1; f += B) assemble_face<kMixed>(cs, f, true);
  const double* __restrict__ x = cs.x;
  double v = 0.0;
  int c = c0 + (int)threadIdx.x;
  if (save_old) {
    double* __restrict__ xo = cs.x_old;
    for (; c < c1; c += B) {
      const double xc = x[c];
      xo[c] = xc;
      v += xc;
    }
  } else {
    for (; c + 3 * B < c1; c += 4 * B) {  // four cells per trip, loads first (fixed order)
      const double a = x[c], b = x[c + B], d = x[c + 2 * B], e = x[c + 3 * B];
      v += a;
      v += b;
      v += d;
      v += e;
    }
    for (; c < c1; c += B) v += x[c];
  }
  return v;
}

// Gauss gradient of T over the cells [c0, c1) into cs.grad (same phase as the sum of T:
// it reads only T and the operator weights).
template <int B, int W>
__device__ __noinline__ void pass_grad(const CaseDev& cs, int c0, int c1) {
  double* __restrict__ G = cs.grad;
  const size_t N = (size_t)cs.N;
  for (int c = c0 + (int)threadIdx.x; c < c1; c += B) {
    double g[3];
    op_grad<W>(cs, c, cs.x, g);
    G[c] = g[0];
    G[N + c] = g[1];
    G[2 * N + c] = g[2];
  }
}

// Pass 2 alone, for matrix read-back (every array of the assembled system written).
template <int B, int W, bool kMixed>
__device__ __noinline__ void pass_rows_only(const CaseDev& cs, int c0, int c1) {
  for (int c = c0 + (int)threadIdx.x; c < c1; c += B)
    store_row<kMixed>(cs, c, assemble_row<W, true>(cs, c, cs.x), true);
}

// ---- L2 prefetch --------------------------------------------------------------------
// The streaming passes request the lines of their next loop trip into L2 before using the
// current one. A prefetch holds no register, so it adds bytes in flight at the 64-register
// occupancy the passes run at. Used where it measured faster: the P and U passes, and the
// row passes of the df64 machinery (lfm_solve_df.cuh); not in A p, whose gathers it slowed.
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// v[c + 2B] and v[c + 3B] (the cells of the next trip of a two-cells-per-trip loop), where
// they are below c1.
template <int B, typename T>
__device__ __forceinline__ void pf_next(const T* v, int c, int c1) {
  if (c + 2 * B < c1) prefetch_l2(v + c + 2 * B);
  if (c + 3 * B < c1) prefetch_l2(v + c + 3 * B);
}

// ---- A v over the slot-major matrix (FP64 or FP32 copy) --------------------------------
template <typename T>
struct Slots {
  int N, W;
  const int32_t* other;  // [W*N] neighbour cell per slot (padding: the cell itself)
  const T* coef;         // [W*N] off-diagonal per slot (padding: 0)
  const T* diag;         // [N]
};

__device__ __forceinline__ Slots<double> slots64(const CaseDev& cs) {
  return Slots<double>{cs.N, cs.W, cs.slot_other, cs.slot_coef, cs.diag};
}
__device__ __forceinline__ Slots<float> slots32(const CaseDev& cs) {
  return Slots<float>{cs.N, cs.W, cs.slot_other, cs.slot_coef32, cs.diag32};
}

__device__ __forceinline__ double fmadd(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmadd(float a, float b, float c) { return fmaf(a, b, c); }

// Rows c and c2 of A v (diag * v_c, then the slots in order, fused multiply-adds), all loads
// of both rows issued before any is used. The matrix arrays are read once per pass with
// evict-first (streaming) loads, so that they do not displace the gathered vector from L1
// and L2.
template <int W, typename T>
__device__ __forceinline__ void rows2(const Slots<T>& A, int c, int c2, const T* __restrict__ v, T& y, T& y2,
                                      T& vc, T& vc2) {
  const size_t N = (size_t)A.N;
  vc = v[c];
  vc2 = v[c2];
  T acc = __ldcs(A.diag + c) * vc, acc2 = __ldcs(A.diag + c2) * vc2;
  if constexpr (W > 0) {
    int o[W], o2[W];
    T u[W], u2[W];
#pragma unroll
    for (int k = 0; k < W; ++k) {
      o[k] = LFM_IDX(__ldcs(A.other + (size_t)k * N + c), A.N, c, kChkSlotCell);
      o2[k] = LFM_IDX(__ldcs(A.other + (size_t)k * N + c2), A.N, c2, kChkSlotCell);
      u[k] = __ldcs(A.coef + (size_t)k * N + c);
      u2[k] = __ldcs(A.coef + (size_t)k * N + c2);
    }
#pragma unroll
    for (int k = 0; k < W; ++k) {
      acc = fmadd(u[k], v[o[k]], acc);
      acc2 = fmadd(u2[k], v[o2[k]], acc2);
    }
  } else {
    for (int k = 0; k < A.W; ++k) {
      const size_t at = (size_t)k * N;
      acc = fmadd(A.coef[at + c], v[LFM_IDX(__ldg(A.other + at + c), A.N, c, kChkSlotCell)], acc);
      acc2 = fmadd(A.coef[at + c2], v[LFM_IDX(__ldg(A.other + at + c2), A.N, c2, kChkSlotCell)], acc2);
    }
  }
  y = acc;
  y2 = acc2;
}

template <int W, typename T>
__device__ __forceinline__ T row1(const Slots<T>& A, int c, const T* __restrict__ v, T& vc) {
  const size_t N = (size_t)A.N;
  const int ns = W > 0 ? W : A.W;
  vc = v[c];
  T acc = A.diag[c] * vc;
#pragma unroll
  for (int k = 0; k < (W > 0 ? W : kMaxSlots); ++k) {
    if (W == 0 && k >= ns) break;
    const size_t at = (size_t)k * N + c;
    acc = fmadd(A.coef[at], v[LFM_IDX(__ldg(A.other + at), A.N, c, kChkSlotCell)], acc);
  }
  return acc;
}

// ---- PCG iteration passes over the cells [c0, c1) of this CTA ---------------------------
// Inlined into the step loop, where the array bases can stay kernel-parameter operands
// (fewer registers held for addresses, more loads in flight). A thread takes cells c and
// c + B per loop trip.

// P: p = w + beta p.
template <int B, typename T>
__device__ __forceinline__ void pass_direction(int c0, int c1, T beta, T* __restrict__ p, const T* __restrict__ w) {
  int c = c0 + (int)threadIdx.x;
  for (; c + B < c1; c += 2 * B) {
    pf_next<B>(p, c, c1);
    pf_next<B>(w, c, c1);
    const T p1 = p[c], p2 = p[c + B], w1 = w[c], w2 = w[c + B];
    p[c] = fmadd(beta, p1, w1);
    p[c + B] = fmadd(beta, p2, w2);
  }
  if (c < c1) p[c] = fmadd(beta, p[c], w[c]);
}

// M (FP64): q = A p; returns this thread's share of p.q.
template <int B, int W>
__device__ __forceinline__ double pass_amul_dot_f64(Slots<double> A, int c0, int c1, const double* __restrict__ p,
                                                 double* __restrict__ q) {
  double s = 0.0;
  int c = c0 + (int)threadIdx.x;
  for (; c + B < c1; c += 2 * B) {
    double y1, y2, pc1, pc2;
    rows2<W>(A, c, c + B, p, y1, y2, pc1, pc2);
    q[c] = y1;
    q[c + B] = y2;
    s = fma(y1, pc1, s);
    s = fma(y2, pc2, s);
  }
  if (c < c1) {
    double pc;
    const double y = row1<W>(A, c, p, pc);
    q[c] = y;
    s = fma(y, pc, s);
  }
  return s;
}

// M (FP32): q = A p; returns this thread's share of p.q, accumulated exactly as FP32 pairs.
template <int B, int W>
__device__ __forceinline__ double pass_amul_dot_f32(Slots<float> A, int c0, int c1, const float* __restrict__ p,
                                                 float* __restrict__ q) {
  Acc2f sig;
  int c = c0 + (int)threadIdx.x;
  for (; c + B < c1; c += 2 * B) {
    float y1, y2, pc1, pc2;
    rows2<W>(A, c, c + B, p, y1, y2, pc1, pc2);
    q[c] = y1;
    q[c + B] = y2;
    sig.add_prod(y1, pc1);
    sig.add_prod(y2, pc2);
  }
  if (c < c1) {
    float pc;
    const float y = row1<W>(A, c, p, pc);
    q[c] = y;
    sig.add_prod(y, pc);
  }
  return sig.value();
}

// ---- M (FP32) with the matrix rows streamed into shared memory by bulk copies ----------
// The CTA's cells go in tiles of 2B, the cells two loop trips of pass_amul_dot_f32 take (a
// thread takes cells j and j + B of a tile). The slot indices, coefficients and diagonal of a
// tile arrive in one of two shared-memory stages (cp.async.bulk, completed on an mbarrier,
// issued by one thread) while the threads work on the other, so the matrix bytes are in
// flight without occupying registers and a thread's global loads are its vector gathers.
// Same cells per thread in the same order, same operations in the same order as the
// register form: equal results bit for bit. Needs N a multiple of 4 (16-byte aligned plane
// starts and tile sizes) and the dynamic shared memory of stage_bytes_f32; ok = false when a
// wait ran out (status recorded; the caller leaves). (The FP64 A p measured slower staged:
// its 8-byte coefficients leave room for one row per thread per tile, or only the indices
// can be staged, and that pass is bound by FP64 issue and the gathers, not by its loads.)
template <int B, int W>
__host__ __device__ constexpr unsigned stage_bytes_f32() {
  return W > 0 ? 2u * (2u * B) * (4u * W + 4u * (W + 1u)) + 16u : 0u;
}

template <int B, int W>
__device__ __forceinline__ bool use_bulk_f32(const Slots<float>& A) {
  return W > 0 && (A.N & 3) == 0 && dyn_smem_bytes() >= stage_bytes_f32<B, W>();
}

template <int B, int W>
__device__ __noinline__ double pass_amul_dot_f32_bulk(Slots<float> A, int c0, int c1, const float* __restrict__ p,
                                                   float* __restrict__ q, const Team& tm, bool& ok) {
  constexpr int TC = 2 * B;
  constexpr int kW = W > 0 ? W : 1;
  constexpr unsigned kPlane = TC * 4u;
  constexpr unsigned kStage = (2u * kW + 1u) * kPlane;
  const size_t N = (size_t)A.N;
  const int tid = threadIdx.x;
  Acc2f sig;
  auto issue = [&](unsigned char* st, int t0, int n, uint64_t* bar, uint64_t pol) {
    const unsigned bytes = (unsigned)n * 4u;
    mbar_arrive_expect_tx(bar, (2u * kW + 1u) * bytes);
#pragma unroll
    for (int k = 0; k < kW; ++k) {
      bulk_g2s(st + k * kPlane, A.other + (size_t)k * N + t0, bytes, bar, pol);
      bulk_g2s(st + (kW + k) * kPlane, A.coef + (size_t)k * N + t0, bytes, bar, pol);
    }
    bulk_g2s(st + 2 * kW * kPlane, A.diag + t0, bytes, bar, pol);
  };
  auto body = [&](const unsigned char* st, int t0, int nt) {
    const int32_t* so = reinterpret_cast<const int32_t*>(st);
    const float* sc = reinterpret_cast<const float*>(st + kW * kPlane);
    const float* sd = reinterpret_cast<const float*>(st + 2 * kW * kPlane);
    const int j = tid;
    if (j + B < nt) {
      // both rows' loads issued before either is used (as in rows2)
      const int j2 = j + B, c = t0 + j, c2 = t0 + j2;
      const float vc = p[c], vc2 = p[c2];
      float acc = sd[j] * vc, acc2 = sd[j2] * vc2;
      int o[kW], o2[kW];
      float u[kW], u2[kW];
#pragma unroll
      for (int k = 0; k < kW; ++k) {
        o[k] = LFM_IDX(so[k * TC + j], A.N, c, kChkSlotCell);
        o2[k] = LFM_IDX(so[k * TC + j2], A.N, c2, kChkSlotCell);
        u[k] = sc[k * TC + j];
        u2[k] = sc[k * TC + j2];
      }
#pragma unroll
      for (int k = 0; k < kW; ++k) {
        acc = fmaf(u[k], p[o[k]], acc);
        acc2 = fmaf(u2[k], p[o2[k]], acc2);
      }
      q[c] = acc;
      q[c2] = acc2;
      sig.add_prod(acc, vc);
      sig.add_prod(acc2, vc2);
    } else if (j < nt) {
      const int c = t0 + j;
      const float vc = p[c];
      float y = sd[j] * vc;
#pragma unroll
      for (int k = 0; k < kW; ++k) y = fmaf(sc[k * TC + j], p[LFM_IDX(so[k * TC + j], A.N, c, kChkSlotCell)], y);
      q[c] = y;
      sig.add_prod(y, vc);
    }
  };
  ok = staged_tiles<TC, kStage>(c0, c1, tm, issue, body);
  return sig.value();
}

// M (FP32) over the bulk-staged rows where the launch gave the shared memory for them, else
// the register form.
template <int B, int W>
__device__ __forceinline__ double amul_dot_f32(Slots<float> A, int c0, int c1, const float* __restrict__ p,
                                               float* __restrict__ q, const Team& tm, bool& ok) {
  ok = true;
  if constexpr (W > 0) {
    if (use_bulk_f32<B, W>(A)) return pass_amul_dot_f32_bulk<B, W>(A, c0, c1, p, q, tm, ok);
  }
  return pass_amul_dot_f32<B, W>(A, c0, c1, p, q);
}

// U (FP64): x += alpha p, r -= alpha q, w = rD r; returns this thread's sum|r| and w.r.
template <int B>
__device__ __forceinline__ double2 pass_update_f64(int c0, int c1, double alpha, double* __restrict__ x,
                                                double* __restrict__ r, double* __restrict__ w,
                                                const double* __restrict__ p, const double* __restrict__ q,
                                                const double* __restrict__ rD) {
  double sa = 0.0, sr = 0.0;
  int c = c0 + (int)threadIdx.x;
  for (; c + B < c1; c += 2 * B) {
    pf_next<B>(p, c, c1);
    pf_next<B>(q, c, c1);
    pf_next<B>(x, c, c1);
    pf_next<B>(r, c, c1);
    pf_next<B>(rD, c, c1);
    const int e = c + B;
    const double pa = p[c], pb = p[e], qa = q[c], qb = q[e];
    const double xa = x[c], xb = x[e], ra = r[c], rb = r[e], da = rD[c], db = rD[e];
    const double rna = fma(-alpha, qa, ra), rnb = fma(-alpha, qb, rb);
    const double wa = da * rna, wb = db * rnb;
    x[c] = fma(alpha, pa, xa);
    x[e] = fma(alpha, pb, xb);
    r[c] = rna;
    r[e] = rnb;
    w[c] = wa;
    w[e] = wb;
    sa += fabs(rna);
    sa += fabs(rnb);
    sr = fma(wa, rna, sr);
    sr = fma(wb, rnb, sr);
  }
  if (c < c1) {
    const double rn = fma(-alpha, q[c], r[c]);
    const double wn = rD[c] * rn;
    x[c] = fma(alpha, p[c], x[c]);
    r[c] = rn;
    w[c] = wn;
    sa += fabs(rn);
    sr = fma(wn, rn, sr);
  }
  return make_double2(sa, sr);
}

// U (FP32 inner solve): dx += a p, r -= a q, w = rD r; returns sum|r| and w.r, each
// accumulated exactly as FP32 pairs. kFirst (the solve's first iteration): dx = a p + 0,
// the same value as dx += a p from the dx = 0 the solve starts from, without reading it (the
// seed passes then need not write that zero).
template <int B, bool kFirst = false>
__device__ __forceinline__ double2 pass_update_f32(int c0, int c1, float a32, float* __restrict__ dx,
                                                float* __restrict__ r, float* __restrict__ w,
                                                const float* __restrict__ p, const float* __restrict__ q,
                                                const float* __restrict__ rD) {
  Acc2f rsum, rho_n;
  int c = c0 + (int)threadIdx.x;
  for (; c + B < c1; c += 2 * B) {
    pf_next<B>(p, c, c1);
    pf_next<B>(q, c, c1);
    if (!kFirst) pf_next<B>(dx, c, c1);
    pf_next<B>(r, c, c1);
    pf_next<B>(rD, c, c1);
    const int e = c + B;
    const float pa = p[c], pb = p[e], qa = q[c], qb = q[e];
    const float xa = kFirst ? 0.0f : dx[c], xb = kFirst ? 0.0f : dx[e], ra = r[c], rb = r[e], da = rD[c],
                db = rD[e];
    const float rna = fmaf(-a32, qa, ra), rnb = fmaf(-a32, qb, rb);
    const float wa = da * rna, wb = db * rnb;
    dx[c] = fmaf(a32, pa, xa);
    dx[e] = fmaf(a32, pb, xb);
    r[c] = rna;
    r[e] = rnb;
    w[c] = wa;
    w[e] = wb;
    rsum.add(fabsf(rna));
    rsum.add(fabsf(rnb));
    rho_n.add_prod(wa, rna);
    rho_n.add_prod(wb, rnb);
  }
  if (c < c1) {
    const float rn = fmaf(-a32, q[c], r[c]);
    const float wn = rD[c] * rn;
    dx[c] = fmaf(a32, p[c], kFirst ? 0.0f : dx[c]);
    r[c] = rn;
    w[c] = wn;
    rsum.add(fabsf(rn));
    rho_n.add_prod(wn, rn);
  }
  return make_double2(rsum.value(), rho_n.value());
}

// Three partial sums of a pass, per thread.
struct Sums3 {
  double a, b, c;
};

// A2 + I (FP64 step): the rows of the matrix and, from the same loaded row, r = b - A x,
// the normFactor terms, sum|r|, w = rD r and rho; p = w. Returns this thread's normFactor
// sum, sum|r| and rho.
template <int B, int W, bool kCorr>
__device__ __noinline__ Sums3 pass_rows_init_f64(const CaseDev& cs, int c0, int c1, double xRef) {
  double* __restrict__ r = cs.r;
  double* __restrict__ p = cs.p;
  const double* __restrict__ x = cs.x;
  double u0 = 0.0, u1 = 0.0, u2 = 0.0;
  for (int c = c0 + (int)threadIdx.x; c < c1; c += B) {
    const Row o = assemble_row<W, kCorr>(cs, c, x);
    const double rd = store_row<false>(cs, c, o, false);
    const double rc = o.s - o.ax;
    u0 += fabs(fma(-o.sa, xRef, o.ax)) + fabs(fma(-o.sa, xRef, o.s));
    u1 += fabs(rc);
    const double wc = rd * rc;
    u2 = fma(wc, rc, u2);
    r[c] = rc;
    p[c] = wc;
  }
  return Sums3{u0, u1, u2};
}

// T (mixed step): the FP64 true residual r = b - A x, rounded to FP32 to seed the inner
// solve (r, w = rD r, p = w; dx starts at zero implicitly: the solve's first update writes it).
// With kFirst it is computed together with the rows of
// the matrix (A2) and the normFactor terms. Returns this thread's normFactor sum (kFirst),
// sum|r| and rho (FP32 terms accumulated exactly as FP32 pairs).
template <int B, int W, bool kFirst, bool kCorr>
__device__ __noinline__ Sums3 pass_true_residual(const CaseDev& cs, int c0, int c1, double xRef) {
  float* __restrict__ r = cs.r32;
  float* __restrict__ w = cs.w32;
  float* __restrict__ p = cs.p32;
  const double* __restrict__ x = cs.x;
  double u0 = 0.0, u1 = 0.0;
  Acc2f rho_acc;
  for (int c = c0 + (int)threadIdx.x; c < c1; c += B) {
    double rc;
    float rd32;
    if (kFirst) {
      const Row o = assemble_row<W, kCorr>(cs, c, x);
      rd32 = (float)store_row<true>(cs, c, o, true);
      u0 += fabs(fma(-o.sa, xRef, o.ax)) + fabs(fma(-o.sa, xRef, o.s));
      rc = o.s - o.ax;
    } else {
      double xc;
      rc = cs.src[c] - row1<W>(slots64(cs), c, x, xc);
      rd32 = cs.rD32[c];
    }
    u1 += fabs(rc);
    const float r32 = (float)rc;
    const float w32 = rd32 * r32;
    rho_acc.add_prod(w32, r32);
    r[c] = r32;
    w[c] = w32;
    p[c] = w32;
  }
  return Sums3{u0, u1, rho_acc.value()};
}

// x += dx (mixed step, FP64).
template <int B>
__device__ __forceinline__ void pass_correct(int c0, int c1, double* __restrict__ x, const float* __restrict__ dx) {
  for (int c = c0 + (int)threadIdx.x; c < c1; c += B) x[c] += (double)dx[c];
}

// Wall time per phase kind, measured by the team's rank-0 thread between barrier exits
// (so each phase's share includes its barrier wait: the team's critical path).
struct PhaseClock {
  bool on;
  unsigned long long t;
  unsigned long long* acc;
  __device__ __forceinline__ PhaseClock(const CaseDev& cs, const Team& tm)
      : on(tm.rank == 0 && threadIdx.x == 0), t(0), acc(cs.sync->phase_ns) {
    if (on) t = global_timer_ns();
  }
  __device__ __forceinline__ void lap(int phase) {
    if (on) {
      const unsigned long long now = global_timer_ns();
      acc[phase] += now - t;
      t = now;
    }
  }
};

__device__ __forceinline__ void write_stats(const CaseDev& cs, const Team& tm, int slot, int iters,
                                            int conv, int sweeps, int status, double init_res,
                                            double final_res, double nf) {
  if (tm.rank == 0 && threadIdx.x == 0) {
    lfm_step_stats st;
    st.iters = iters;
    st.converged = conv;
    st.sweeps = sweeps;
    st.status = status;
    st.init_res = init_res;
    st.final_res = final_res;
    st.norm_factor = nf;
    cs.stats[slot] = st;
  }
}

// Start of an assembly: the per-thread sums of T (with the faces for matrix read-back, the
// copy of T at the start of the step when save_old, and with general geometry the Gauss
// gradient in the same phase) and their team sum for xRef. False when a barrier failed (the
// caller leaves the kernel).
template <int B, int W, bool kMixed>
__device__ __forceinline__ bool assemble_prologue(const CaseDev& cs, const CaseDev& cref, const Team& tm, int c0,
                                                  int c1, int f0, int f1, bool write_upper, bool save_old,
                                                  double& sum_x, TeamShared& sh) {
  double v[1] = {pass_faces<B, kMixed>(cref, f0, f1, c0, c1, write_upper, save_old)};
  if (cs.Sf) pass_grad<B, W>(cref, c0, c1);
  if (!team_allreduce<1>(tm, v, sh)) return false;
  sum_x = v[0];
  return true;
}

// =======================================================================================
// FP64 steps (1 + n_corr assemble-and-solve passes per step)
// =======================================================================================
template <int B, int W>
__device__ void run_steps_f64(const CaseDev& cs, const CaseDev& cref, const Team& tm, int n_steps, int mode,
                              TeamShared& sh,
                              int stats_base = 0) {
  int c0, c1, f0, f1;
  cta_range(cs.N, tm.size, tm.rank, c0, c1);
  cta_range(cs.F, tm.size, tm.rank, f0, f1);
  const int tid = threadIdx.x;
  double* __restrict__ x = cs.x;
  double* __restrict__ r = cs.r;
  double* __restrict__ w = cs.w;
  double* __restrict__ p = cs.p;
  double* __restrict__ q = cs.q;
  const double* __restrict__ rD = cs.rD;

  PhaseClock clk(cs, tm);
  const bool corr_mode = cs.n_corr > 0 || cs.Sf != nullptr || cs.vSu != nullptr || cs.vSp != nullptr;
  for (int step = 0; step < n_steps; ++step) {
    int iters_tot = 0, solves = 0, status = 0;
    double nf0 = 0.0, init0 = 0.0, res = 0.0;
    bool conv = false;
    for (int pass = 0; pass <= cs.n_corr; ++pass) {
      // ---- A1: face coefficients, sum of T (and the gradient / correction fluxes) --------
      double sum_x = 0.0;
      if (!assemble_prologue<B, W, false>(cs, cref, tm, c0, c1, f0, f1, mode == kModeAssembleOnly,
                                       pass == 0 && cs.n_corr > 0, sum_x, sh))
        return;
      clk.lap(kPhAssembly);
      if (mode == kModeAssembleOnly) {
        pass_rows_only<B, W, false>(cref, c0, c1);
        return;
      }
      // ---- A2 + I: rows of the matrix, initial residual, normFactor, first direction -----
      const double xRef = sum_x / (double)cs.N;
      const Sums3 ui = corr_mode ? pass_rows_init_f64<B, W, true>(cref, c0, c1, xRef)
                                 : pass_rows_init_f64<B, W, false>(cref, c0, c1, xRef);
      double u[3] = {ui.a, ui.b, ui.c};  // normFactor sum, sum|r|, rho
      if (!team_allreduce<3>(tm, u, sh)) return;
      clk.lap(kPhInit);
      const double nf = u[0] + kSmall;
      const double init_res = u[1] / nf;
      res = init_res;
      double rho = u[2], beta = 0.0;
      int iters = 0;
      conv = converged(res, init_res, cs.tol, cs.rel_tol);
      if (cs.min_iter > 0 || !conv) {
        for (;;) {
          if (iters > 0) {
            // ---- P: search direction -----------------------------------------------
            pass_direction<B, double>(c0, c1, beta, p, w);
            if (!team_barrier(tm, sh)) return;
            clk.lap(kPhP);
          }
          // ---- M: q = A p, sigma = p.q --------------------------------------------
          double s1[1] = {pass_amul_dot_f64<B, W>(slots64(cs), c0, c1, p, q)};
          if (!team_allreduce<1>(tm, s1, sh)) return;
          clk.lap(kPhM);
          const double sigma = s1[0];
          if (fabs(sigma) / nf < kVSmall) {
            status = LFM_ESINGULAR;
            break;
          }
          const double alpha = rho / sigma;
          // ---- U: update, residual, preconditioned residual, next rho --------------
          const double2 su = pass_update_f64<B>(c0, c1, alpha, x, r, w, p, q, rD);
          double s2[2] = {su.x, su.y};
          if (!team_allreduce<2>(tm, s2, sh)) return;
          clk.lap(kPhU);
          res = s2[0] / nf;
          beta = s2[1] / rho;
          rho = s2[1];
          ++iters;
          if (!isfinite(res)) {
            status = LFM_ENONFINITE;
            break;
          }
          conv = converged(res, init_res, cs.tol, cs.rel_tol);
          if (!((iters < cs.max_iter && !conv) || iters < cs.min_iter)) break;
        }
      }
      conv = converged(res, init_res, cs.tol, cs.rel_tol);
      if (pass == 0) {
        nf0 = nf;
        init0 = init_res;
      }
      iters_tot += iters;
      solves += iters > 0 ? 1 : 0;
      if (status != 0) break;
    }
    write_stats(cs, tm, stats_base + step, iters_tot, conv ? 1 : 0, solves, status, init0, res, nf0);
    if (status != 0) {
      if (tm.rank == 0 && tid == 0) set_status(cs.sync, status);
      return;
    }
  }
}

// =======================================================================================
// Mixed-precision steps (FP32 inner CG inside FP64 defect correction)
// =======================================================================================
template <int B, int W>
__device__ void run_steps_mixed(const CaseDev& cs, const CaseDev& cref, const Team& tm, int n_steps, int mode,
                              TeamShared& sh,
                                int stats_base = 0) {
  int c0, c1, f0, f1;
  cta_range(cs.N, tm.size, tm.rank, c0, c1);
  cta_range(cs.F, tm.size, tm.rank, f0, f1);
  const int tid = threadIdx.x;
  double* __restrict__ x = cs.x;
  float* __restrict__ dx = cs.dx32;
  float* __restrict__ r = cs.r32;
  float* __restrict__ w = cs.w32;
  float* __restrict__ p = cs.p32;
  float* __restrict__ q = cs.q32;
  const float* __restrict__ rD = cs.rD32;

  PhaseClock clk(cs, tm);
  const bool corr_mode = cs.n_corr > 0 || cs.Sf != nullptr || cs.vSu != nullptr || cs.vSp != nullptr;
  for (int step = 0; step < n_steps; ++step) {
    int iters_tot = 0, sweeps_tot = 0, status = 0;
    double nf0 = 0.0, init0 = 0.0, res = 0.0;
    bool conv = false;
    for (int pass = 0; pass <= cs.n_corr; ++pass) {
      double sum_x = 0.0;
      if (!assemble_prologue<B, W, true>(cs, cref, tm, c0, c1, f0, f1, mode == kModeAssembleOnly,
                                      pass == 0 && cs.n_corr > 0, sum_x, sh))
        return;
      clk.lap(kPhAssembly);
      if (mode == kModeAssembleOnly) {
        pass_rows_only<B, W, true>(cref, c0, c1);
        return;
      }
      const double xRef = sum_x / (double)cs.N;

      double nf = 0.0, init_res = 0.0;
      int iters = 0, sweeps = 0;
      for (;;) {
        // ---- T: FP64 true residual r = b - A x, seeded into the FP32 inner solve; on the
        //      first sweep computed together with pass 2 of the assembly and normFactor ---
        Sums3 ui;
        if (sweeps > 0)
          ui = pass_true_residual<B, W, false, false>(cref, c0, c1, xRef);
        else if (corr_mode)
          ui = pass_true_residual<B, W, true, true>(cref, c0, c1, xRef);
        else
          ui = pass_true_residual<B, W, true, false>(cref, c0, c1, xRef);
        double u[3] = {ui.a, ui.b, ui.c};  // normFactor sum (first sweep), sum|r|, rho
        if (!team_allreduce<3>(tm, u, sh)) return;
        clk.lap(kPhInit);
        if (sweeps == 0) {
          nf = u[0] + kSmall;
          init_res = u[1] / nf;
        }
        res = u[1] / nf;
        if (!isfinite(res)) {
          status = LFM_ENONFINITE;
          break;
        }
        const bool c_ok = converged(res, init_res, cs.tol, cs.rel_tol);
        if ((c_ok && !(sweeps == 0 && cs.min_iter > 0)) || sweeps == kMaxSweeps || iters >= cs.max_iter) break;

        // ---- inner FP32 CG on A dx = r ------------------------------------------------
        const double inner_tol = fmax(cs.tol, kInnerRel * res);
        const int min_inner = sweeps == 0 ? cs.min_iter : 0;
        double rho = u[2], beta = 0.0;
        int k = 0;
        for (;;) {
          if (k > 0) {
            pass_direction<B, float>(c0, c1, (float)beta, p, w);
            if (!team_barrier(tm, sh)) return;
            clk.lap(kPhP);
          }
          bool m_ok;
          double s1[1] = {amul_dot_f32<B, W>(slots32(cs), c0, c1, p, q, tm, m_ok)};
          if (!m_ok) return;
          if (!team_allreduce<1>(tm, s1, sh)) return;
          clk.lap(kPhM);
          const double sigma = s1[0];
          if (fabs(sigma) / nf < kVSmall) {
            status = LFM_ESINGULAR;
            break;
          }
          const double2 su = k == 0 ? pass_update_f32<B, true>(c0, c1, (float)(rho / sigma), dx, r, w, p, q, rD)
                                    : pass_update_f32<B, false>(c0, c1, (float)(rho / sigma), dx, r, w, p, q, rD);
          double s2[2] = {su.x, su.y};
          if (!team_allreduce<2>(tm, s2, sh)) return;
          clk.lap(kPhU);
          const double inner_res = s2[0] / nf;
          beta = s2[1] / rho;
          rho = s2[1];
          ++k;
          ++iters;
          if (!isfinite(inner_res)) {
            status = LFM_ENONFINITE;
            break;
          }
          const bool inner_conv = inner_res < inner_tol;
          if (!((iters < cs.max_iter && !inner_conv) || k < min_inner)) break;
        }
        if (status != 0) break;
        // ---- x += dx (FP64) ----------------------------------------------------------
        pass_correct<B>(c0, c1, x, dx);
        if (!team_barrier(tm, sh)) return;
        clk.lap(kPhCorrect);
        ++sweeps;
      }
      conv = converged(res, init_res, cs.tol, cs.rel_tol);
      if (pass == 0) {
        nf0 = nf;
        init0 = init_res;
      }
      iters_tot += iters;
      sweeps_tot += sweeps;
      if (status != 0) break;
    }
    write_stats(cs, tm, stats_base + step, iters_tot, conv ? 1 : 0, sweeps_tot, status, init0, res, nf0);
    if (status != 0) {
      if (tm.rank == 0 && tid == 0) set_status(cs.sync, status);
      return;
    }
  }
}

}  // namespace
}  // namespace lfm

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
// FP64 step (phases separated by team barriers):
//   A  assembly        per slot g = DT |Sf| deltaCoeff; diag, the per-slot off-diagonals
//                      (each face's coefficient at both of its cells; the face-indexed
//                      LDU `upper` is written only for matrix read-back), source,
//                      rD = 1/diag, row sums; sum x for xRef
//   I  initial state   A x, r = b - A x, row sums -> normFactor, sum|r|, w = rD r, rho;
//                      p = w (first search direction)
//   loop (diagonal-preconditioned CG, convergence on sum|r| / normFactor):
//   P  p = w + beta p  (skipped on the first iteration)
//   M  q = A p, sigma = p.q                   -> alpha = rho / sigma
//   U  x += alpha p, r -= alpha q, w = rD r, sum|r|, rho' = w.r -> beta = rho'/rho
//
// Mixed step (defect correction, FP64 field x): the matrix is assembled in FP64 and copied
// to FP32; each sweep computes the FP64 true residual r = b - A x, solves A dx = r by the
// same CG recurrence on FP32 vectors with FP32 row sums, and adds dx to x in FP64. Dot
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

// ---- assembly of fvm::ddt(T) - fvm::laplacian(DT, T), two passes ---------------------
// Pass 1 (per cell, its owned faces): g = (DT |Sf|) deltaCoeff, computed once per face and
// stored as -g in the cell's slot and in the neighbour's matching slot (slot_mate).
template <bool kMixed>
__device__ __forceinline__ void assemble_faces(const CaseDev& cs, int c, int ns, bool write_upper) {
  const size_t N = (size_t)cs.N;
  for (int k = 0; k < ns; ++k) {
    const size_t at = (size_t)k * N + c;
    const int mate = __ldg(cs.slot_mate + at);
    if (mate >= 0) {
      const int f = __ldg(cs.slot_face + at);
      const int n = __ldg(cs.slot_other + at);
      const double DTf = cs.DT_is_uniform ? cs.DT_uniform : __ldg(cs.DT + f);
      const double g = __dmul_rn(__dmul_rn(DTf, __ldg(cs.magSf + f)), __ldg(cs.delta + f));
      const size_t at_n = (size_t)mate * N + n;
      cs.slot_coef[at] = -g;
      cs.slot_coef[at_n] = -g;
      if (kMixed) {
        cs.slot_coef32[at] = (float)(-g);
        cs.slot_coef32[at_n] = (float)(-g);
      }
      if (write_upper) cs.upper[f] = -g;  // the face-indexed LDU copy, for read-back only
    }
  }
}

// Pass 2 (per cell): the diagonal summed in slot order, i.e. ascending face order
// (neighbour-side faces have smaller owners, so they precede the cell's own faces in
// upper-triangular order), then the boundary faces, then V/dt; every product and sum rounded
// separately (no FMA); source, 1/diag and the row sum. Returns the cell's T.
template <int W, bool kMixed>
__device__ __forceinline__ double assemble_diag(const CaseDev& cs, int c) {
  const size_t N = (size_t)cs.N;
  const int ns = nslots<W>(cs);
  double d = 0.0, s = 0.0;
#pragma unroll
  for (int k = 0; k < (W > 0 ? W : kMaxSlots); ++k) {
    if (W == 0 && k >= ns) break;
    d = __dadd_rn(d, -cs.slot_coef[(size_t)k * N + c]);  // padding slots hold 0
  }
  double gsum = 0.0;  // boundary conductance of the row
  const int b0 = __ldg(cs.b_start + c), b1 = __ldg(cs.b_start + c + 1);
  for (int k = b0; k < b1; ++k) {
    const int bf = __ldg(cs.b_face + k);
    if (__ldg(cs.btype + bf) == LFM_FIXED_VALUE) {
      const double gb = __dmul_rn(__dmul_rn(__ldg(cs.bDT + bf), __ldg(cs.bmagSf + bf)), __ldg(cs.bdelta + bf));
      d = __dadd_rn(d, gb);
      s = __dadd_rn(s, __dmul_rn(gb, __ldg(cs.bval + bf)));
      gsum = __dadd_rn(gsum, gb);
    }
  }
  const double vdt = cs.vdt[c];  // V/dt, hoisted out of the time loop (same IEEE quotient)
  const double xc = cs.x[c];
  d = __dadd_rn(d, vdt);
  s = __dadd_rn(s, __dmul_rn(vdt, xc));
  const double rd = __drcp_rn(d);  // IEEE round-to-nearest reciprocal, as 1.0 / d
  cs.diag[c] = d;
  cs.src[c] = s;
  cs.rD[c] = rd;
  // Row sum of A: the off-diagonals cancel the face conductances in the diagonal exactly in
  // real arithmetic, leaving V/dt plus the boundary conductance.
  cs.sumA[c] = gsum + vdt;
  if (kMixed) {
    cs.diag32[c] = (float)d;
    cs.rD32[c] = (float)rd;
  }
  return xc;
}

// Both passes for this CTA's cells, with the team barrier between them. v0 receives the
// CTA threads' sum of T (for xRef); false when a barrier failed.
template <int B, int W, bool kMixed>
__device__ __forceinline__ bool assemble(const CaseDev& cs, const Team& tm, int c0, int c1, bool write_upper,
                                         double& sum_x, TeamShared& sh) {
  const int ns = nslots<W>(cs);
  for (int c = c0 + (int)threadIdx.x; c < c1; c += B) assemble_faces<kMixed>(cs, c, ns, write_upper);
  if (!team_barrier(tm, sh)) return false;
  double v = 0.0;
  for (int c = c0 + (int)threadIdx.x; c < c1; c += B) v += assemble_diag<W, kMixed>(cs, c);
  sum_x = v;
  return true;
}

// ---- FP64 A v for two rows at once (FMA accumulation) ----------------------------------
template <int W>
__device__ __forceinline__ void rows2_f64(const CaseDev& cs, int c, int c2, const double* __restrict__ v,
                                          double& y, double& y2, double& vc, double& vc2) {
  const size_t N = (size_t)cs.N;
  vc = v[c];
  vc2 = v[c2];
  double acc = cs.diag[c] * vc, acc2 = cs.diag[c2] * vc2;
  if constexpr (W > 0) {
    int o[W], o2[W];
    double u[W], u2[W];
#pragma unroll
    for (int k = 0; k < W; ++k) {
      o[k] = __ldg(cs.slot_other + (size_t)k * N + c);
      o2[k] = __ldg(cs.slot_other + (size_t)k * N + c2);
      u[k] = cs.slot_coef[(size_t)k * N + c];
      u2[k] = cs.slot_coef[(size_t)k * N + c2];
    }
#pragma unroll
    for (int k = 0; k < W; ++k) {
      acc = fma(u[k], v[o[k]], acc);
      acc2 = fma(u2[k], v[o2[k]], acc2);
    }
  } else {
    const int ns = cs.W;
    for (int k = 0; k < ns; ++k) {
      const size_t at = (size_t)k * N;
      acc = fma(cs.slot_coef[at + c], v[__ldg(cs.slot_other + at + c)], acc);
      acc2 = fma(cs.slot_coef[at + c2], v[__ldg(cs.slot_other + at + c2)], acc2);
    }
  }
  y = acc;
  y2 = acc2;
}

template <int W>
__device__ __forceinline__ double row_f64(const CaseDev& cs, int c, const double* __restrict__ v, double& vc) {
  const size_t N = (size_t)cs.N;
  const int ns = nslots<W>(cs);
  vc = v[c];
  double acc = cs.diag[c] * vc;
#pragma unroll
  for (int k = 0; k < (W > 0 ? W : kMaxSlots); ++k) {
    if (W == 0 && k >= ns) break;
    const size_t at = (size_t)k * N + c;
    acc = fma(cs.slot_coef[at], v[__ldg(cs.slot_other + at)], acc);
  }
  return acc;
}

// ---- FP32 A v --------------------------------------------------------------------------
template <int W>
__device__ __forceinline__ void rows2_f32(const CaseDev& cs, int c, int c2, const float* __restrict__ v,
                                          float& y, float& y2, float& vc, float& vc2) {
  const size_t N = (size_t)cs.N;
  vc = v[c];
  vc2 = v[c2];
  float acc = cs.diag32[c] * vc, acc2 = cs.diag32[c2] * vc2;
  if constexpr (W > 0) {
    int o[W], o2[W];
    float u[W], u2[W];
#pragma unroll
    for (int k = 0; k < W; ++k) {
      o[k] = __ldg(cs.slot_other + (size_t)k * N + c);
      o2[k] = __ldg(cs.slot_other + (size_t)k * N + c2);
      u[k] = cs.slot_coef32[(size_t)k * N + c];
      u2[k] = cs.slot_coef32[(size_t)k * N + c2];
    }
#pragma unroll
    for (int k = 0; k < W; ++k) {
      acc = fmaf(u[k], v[o[k]], acc);
      acc2 = fmaf(u2[k], v[o2[k]], acc2);
    }
  } else {
    const int ns = cs.W;
    for (int k = 0; k < ns; ++k) {
      const size_t at = (size_t)k * N;
      acc = fmaf(cs.slot_coef32[at + c], v[__ldg(cs.slot_other + at + c)], acc);
      acc2 = fmaf(cs.slot_coef32[at + c2], v[__ldg(cs.slot_other + at + c2)], acc2);
    }
  }
  y = acc;
  y2 = acc2;
}

template <int W>
__device__ __forceinline__ float row_f32(const CaseDev& cs, int c, const float* __restrict__ v, float& vc) {
  const size_t N = (size_t)cs.N;
  const int ns = nslots<W>(cs);
  vc = v[c];
  float acc = cs.diag32[c] * vc;
#pragma unroll
  for (int k = 0; k < (W > 0 ? W : kMaxSlots); ++k) {
    if (W == 0 && k >= ns) break;
    const size_t at = (size_t)k * N + c;
    acc = fmaf(cs.slot_coef32[at], v[__ldg(cs.slot_other + at)], acc);
  }
  return acc;
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

// =======================================================================================
// FP64 steps
// =======================================================================================
template <int B, int W>
__device__ void run_steps_f64(const CaseDev& cs, const Team& tm, int n_steps, int mode, TeamShared& sh,
                              int stats_base = 0) {
  int c0, c1;
  cta_range(cs.N, tm.size, tm.rank, c0, c1);
  const int tid = threadIdx.x;
  double* __restrict__ x = cs.x;
  double* __restrict__ r = cs.r;
  double* __restrict__ w = cs.w;
  double* __restrict__ p = cs.p;
  double* __restrict__ q = cs.q;
  const double* __restrict__ rD = cs.rD;

  PhaseClock clk(cs, tm);
  for (int step = 0; step < n_steps; ++step) {
    // ---- A: assembly ---------------------------------------------------------------------
    double v[1] = {0.0};
    if (!assemble<B, W, false>(cs, tm, c0, c1, mode == kModeAssembleOnly, v[0], sh)) return;
    if (!team_allreduce<1>(tm, v, sh)) return;
    clk.lap(kPhAssembly);
    if (mode == kModeAssembleOnly) return;
    // ---- I: initial residual, normFactor, first direction -----------------------------
    const double xRef = v[0] / (double)cs.N;
    double u[3] = {0.0, 0.0, 0.0};  // normFactor sum, sum|r|, rho
    for (int c = c0 + tid; c < c1; c += B) {
      const double b = cs.src[c];
      double xc;
      const double ax = row_f64<W>(cs, c, x, xc);
      const double rc = b - ax;
      const double pA = cs.sumA[c] * xRef;
      u[0] += fabs(ax - pA) + fabs(b - pA);
      u[1] += fabs(rc);
      const double wc = rD[c] * rc;
      u[2] = fma(wc, rc, u[2]);
      r[c] = rc;
      p[c] = wc;
    }
    if (!team_allreduce<3>(tm, u, sh)) return;
    clk.lap(kPhInit);
    const double nf = u[0] + kSmall;
    const double init_res = u[1] / nf;
    double res = init_res, rho = u[2], beta = 0.0;
    int iters = 0, status = 0;
    bool conv = converged(res, init_res, cs.tol, cs.rel_tol);
    if (cs.min_iter > 0 || !conv) {
      for (;;) {
        if (iters > 0) {
          // ---- P: search direction -------------------------------------------------
          int c = c0 + tid;
          for (; c + B < c1; c += 2 * B) {
            const double p1 = p[c], p2 = p[c + B], w1 = w[c], w2 = w[c + B];
            p[c] = fma(beta, p1, w1);
            p[c + B] = fma(beta, p2, w2);
          }
          if (c < c1) p[c] = fma(beta, p[c], w[c]);
          if (!team_barrier(tm, sh)) return;
          clk.lap(kPhP);
        }
        // ---- M: q = A p, sigma = p.q ----------------------------------------------
        double s1[1] = {0.0};
        {
          int c = c0 + tid;
          for (; c + B < c1; c += 2 * B) {
            double y1, y2, pc1, pc2;
            rows2_f64<W>(cs, c, c + B, p, y1, y2, pc1, pc2);
            q[c] = y1;
            q[c + B] = y2;
            s1[0] = fma(y1, pc1, s1[0]);
            s1[0] = fma(y2, pc2, s1[0]);
          }
          if (c < c1) {
            double pc;
            const double y = row_f64<W>(cs, c, p, pc);
            q[c] = y;
            s1[0] = fma(y, pc, s1[0]);
          }
        }
        if (!team_allreduce<1>(tm, s1, sh)) return;
        clk.lap(kPhM);
        const double sigma = s1[0];
        if (fabs(sigma) / nf < kVSmall) {
          status = LFM_ESINGULAR;
          break;
        }
        const double alpha = rho / sigma;
        // ---- U: update, residual, preconditioned residual, next rho ----------------
        double s2[2] = {0.0, 0.0};
        {
          int c = c0 + tid;
          for (; c + B < c1; c += 2 * B) {
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
            s2[0] += fabs(rna);
            s2[0] += fabs(rnb);
            s2[1] = fma(wa, rna, s2[1]);
            s2[1] = fma(wb, rnb, s2[1]);
          }
          if (c < c1) {
            const double rn = fma(-alpha, q[c], r[c]);
            const double wn = rD[c] * rn;
            x[c] = fma(alpha, p[c], x[c]);
            r[c] = rn;
            w[c] = wn;
            s2[0] += fabs(rn);
            s2[1] = fma(wn, rn, s2[1]);
          }
        }
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
    write_stats(cs, tm, stats_base + step, iters, conv ? 1 : 0, iters > 0 ? 1 : 0, status, init_res, res, nf);
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
__device__ void run_steps_mixed(const CaseDev& cs, const Team& tm, int n_steps, int mode, TeamShared& sh,
                                int stats_base = 0) {
  int c0, c1;
  cta_range(cs.N, tm.size, tm.rank, c0, c1);
  const int tid = threadIdx.x;
  double* __restrict__ x = cs.x;
  float* __restrict__ dx = cs.dx32;
  float* __restrict__ r = cs.r32;
  float* __restrict__ w = cs.w32;
  float* __restrict__ p = cs.p32;
  float* __restrict__ q = cs.q32;
  const float* __restrict__ rD = cs.rD32;

  PhaseClock clk(cs, tm);
  for (int step = 0; step < n_steps; ++step) {
    double v[1] = {0.0};
    if (!assemble<B, W, true>(cs, tm, c0, c1, mode == kModeAssembleOnly, v[0], sh)) return;
    if (!team_allreduce<1>(tm, v, sh)) return;
    clk.lap(kPhAssembly);
    if (mode == kModeAssembleOnly) return;
    const double xRef = v[0] / (double)cs.N;

    double nf = 0.0, init_res = 0.0, res = 0.0;
    int iters = 0, sweeps = 0, status = 0;
    for (;;) {
      // ---- T: FP64 true residual r = b - A x, seeded into the FP32 inner solve --------
      double u[3] = {0.0, 0.0, 0.0};  // normFactor sum (first sweep), sum|r|, rho
      Acc2f rho_acc;
      for (int c = c0 + tid; c < c1; c += B) {
        const double b = cs.src[c];
        double xc;
        const double ax = row_f64<W>(cs, c, x, xc);
        const double rc = b - ax;
        if (sweeps == 0) {
          const double pA = cs.sumA[c] * xRef;
          u[0] += fabs(ax - pA) + fabs(b - pA);
        }
        u[1] += fabs(rc);
        const float r32 = (float)rc;
        const float w32 = rD[c] * r32;
        rho_acc.add_prod(w32, r32);
        r[c] = r32;
        w[c] = w32;
        p[c] = w32;
        dx[c] = 0.0f;
      }
      u[2] = rho_acc.value();
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
      const bool conv = converged(res, init_res, cs.tol, cs.rel_tol);
      if ((conv && !(sweeps == 0 && cs.min_iter > 0)) || sweeps == kMaxSweeps || iters >= cs.max_iter) break;

      // ---- inner FP32 CG on A dx = r --------------------------------------------------
      const double inner_tol = fmax(cs.tol, kInnerRel * res);
      const int min_inner = sweeps == 0 ? cs.min_iter : 0;
      double rho = u[2], beta = 0.0;
      int k = 0;
      for (;;) {
        if (k > 0) {
          const float b32 = (float)beta;
          int c = c0 + tid;
          for (; c + B < c1; c += 2 * B) {
            const float p1 = p[c], p2 = p[c + B], w1 = w[c], w2 = w[c + B];
            p[c] = fmaf(b32, p1, w1);
            p[c + B] = fmaf(b32, p2, w2);
          }
          if (c < c1) p[c] = fmaf(b32, p[c], w[c]);
          if (!team_barrier(tm, sh)) return;
          clk.lap(kPhP);
        }
        double s1[1];
        {
          Acc2f sig;
          int c = c0 + tid;
          for (; c + B < c1; c += 2 * B) {
            float y1, y2, pc1, pc2;
            rows2_f32<W>(cs, c, c + B, p, y1, y2, pc1, pc2);
            q[c] = y1;
            q[c + B] = y2;
            sig.add_prod(y1, pc1);
            sig.add_prod(y2, pc2);
          }
          if (c < c1) {
            float pc;
            const float y = row_f32<W>(cs, c, p, pc);
            q[c] = y;
            sig.add_prod(y, pc);
          }
          s1[0] = sig.value();
        }
        if (!team_allreduce<1>(tm, s1, sh)) return;
        clk.lap(kPhM);
        const double sigma = s1[0];
        if (fabs(sigma) / nf < kVSmall) {
          status = LFM_ESINGULAR;
          break;
        }
        const float a32 = (float)(rho / sigma);
        double s2[2];
        {
          Acc2f rsum, rho_n;
          int c = c0 + tid;
          for (; c + B < c1; c += 2 * B) {
            const int e = c + B;
            const float pa = p[c], pb = p[e], qa = q[c], qb = q[e];
            const float xa = dx[c], xb = dx[e], ra = r[c], rb = r[e], da = rD[c], db = rD[e];
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
            dx[c] = fmaf(a32, p[c], dx[c]);
            r[c] = rn;
            w[c] = wn;
            rsum.add(fabsf(rn));
            rho_n.add_prod(wn, rn);
          }
          s2[0] = rsum.value();
          s2[1] = rho_n.value();
        }
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
      // ---- x += dx (FP64) ------------------------------------------------------------
      for (int c = c0 + tid; c < c1; c += B) x[c] += (double)dx[c];
      if (!team_barrier(tm, sh)) return;
      clk.lap(kPhCorrect);
      ++sweeps;
    }
    const bool conv = converged(res, init_res, cs.tol, cs.rel_tol);
    write_stats(cs, tm, stats_base + step, iters, conv ? 1 : 0, sweeps, status, init_res, res, nf);
    if (status != 0) {
      if (tm.rank == 0 && tid == 0) set_status(cs.sync, status);
      return;
    }
  }
}

}  // namespace
}  // namespace lfm

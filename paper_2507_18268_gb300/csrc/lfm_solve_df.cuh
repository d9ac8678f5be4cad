// lfm_solve_df.cuh -- the implicit laplacianFoam step in df64 (double-float) arithmetic,
// shared by the single-case kernel (lfm_step.cu) and the batched kernel (lfm_batch.cu).
//
// The same method as the FP64 step in lfm_solve.cuh (Eq. (1), the listing "laplacianFoam
// application": per step assemble fvm::ddt(T) - fvm::laplacian(DT, T) and solve it with the
// diagonal-preconditioned CG, convergence on OpenFOAM's normFactor-scaled L1 residual), with
// every per-cell operation done in df64 on the FP32 pipe (lfm_df64.cuh) and only per-CTA
// scalars (alpha, beta, the reduced sums) in FP64. Storage is 8 bytes per value as in FP64.
//
// Set-up (a0, when the mesh, DT or dt change): the face conductances g_f = DT_f |S_f|
// deltaCoeff_f, formed in FP64, are stored per slot as df64 (g2, the face's value at its
// slot in both of its cells' rows), and V/dt per cell (vdt2). Both are multiplied by the
// case's power-of-two scale s (df_scale), chosen so that V/dt is of order one: PCG is
// invariant under scaling A and b by a common factor, a power of two scales every FP64
// and df64 value exactly, and the scaled values keep far from FP32's underflow. Reported
// normFactors are divided by s.
//
// Per launch: the field T (FP64, x) is split into a triple-float (x2 = hi, mid; xlo = lo;
// see lfm_df64.cuh) by the first pass when x was written since the last df64 launch (flags),
// and its rounding is written back to x after the last step; otherwise the triple-float field
// carries over from the previous launch, so that launch boundaries do not round the field. Fluxes and
// ddt terms are differences of field values formed exactly from the three parts, and the
// per-iteration update adds the df64 correction to all three, so rounding at df64's 2^-48 is
// relative to corrections and differences, never to T itself. (A per-step rounding of T to
// 48 bits is a noise source that truncated-CG time stepping amplifies from step to step:
// on the 200^3 graded box it grew to 7e-10 relative over 100 steps.)
// Per step (phases separated by team barriers):
//   S  the last solve's correction added to the field; sum of x (for xRef); with correctors
//      also x at the start of the step
//   R  per row: diag = sum of the slot conductances (slot order) + boundary + V/dt, the
//      source, 1/diag (FP32 reciprocal + one df64 Newton step), the row sum; r = b - A x
//      (in flux form, see pass_rows_init_df), normFactor terms, sum|r|, w = rD r, rho; p = w
//   loop: P p = w + beta p; M q = A p, p.q; U e += alpha p, r -= alpha q, w = rD r, sum|r|, w.r
//   (e: the solve's correction to the field, df64)
// A row of A v is diag_c v_c - sum_k g_ck v_other(k): the off-diagonal coefficient of face f
// is -g_f in both rows (the matrix is symmetric), so the slot array of conductances is the
// matrix's off-diagonal part.
//
// Boundary faces (a few per cent of cells) are summed in FP64 and converted once per row;
// so are the optional volumetric sources. On general (non-orthogonal) geometry (kGeom) a
// phase G after S forms the Gauss gradient of the field and R adds the explicit correction.
// The mixed form's df64 outer passes are in lfm_solve_mixed_df.cuh.
#pragma once

#include <cuda_runtime.h>

#include "lfm_device.cuh"
#include "lfm_df64.cuh"
#include "lfm_internal.h"
#include "lfm_solve.cuh"

namespace lfm {
namespace {

__device__ __forceinline__ df df_from_scalar(double v) { return df_from_double(v); }

// S: this thread's sum of x over [c0, c1) (per-thread df64 sum, converted once). `convert`:
// first pass of the launch, the triple-float field is split from the FP64 field x. `fold`:
// the previous solve's correction e (df64, see pass_update_df) is added to the field first.
// `save_old`: keep x as the step's starting field (the ddt source of the corrector passes).
template <int B>
__device__ __noinline__ double pass_sum_df(const CaseDev& cs, int c0, int c1, bool convert, bool fold,
                                           bool save_old) {
  float2* __restrict__ x2 = cs.x2;
  float* __restrict__ xl = cs.xlo;
  const float2* __restrict__ e2 = cs.e2;
  DfAcc acc;
  int c = c0 + (int)threadIdx.x;
  if (!convert && !save_old) {  // two cells per trip, loads first
    for (; c + B < c1; c += 2 * B) {
      tf a = ld_tf(x2, xl, c), b = ld_tf(x2, xl, c + B);
      if (fold) {
        const df ea = ld_df(e2 + c), eb = ld_df(e2 + c + B);
        a = tf_add_df(a, ea);
        b = tf_add_df(b, eb);
        st_tf(x2, xl, c, a);
        st_tf(x2, xl, c + B, b);
      }
      acc.add(tf_to_df(a));
      acc.add(tf_to_df(b));
    }
  }
  for (; c < c1; c += B) {
    tf v;
    if (convert) {
      v = tf_from_double(cs.x[c]);
      st_tf(x2, xl, c, v);
    } else {
      v = ld_tf(x2, xl, c);
      if (fold) {
        v = tf_add_df(v, ld_df(e2 + c));
        st_tf(x2, xl, c, v);
      }
    }
    if (save_old) st_tf(reinterpret_cast<float2*>(cs.x_old), cs.xolo, c, v);
    acc.add(tf_to_df(v));
  }
  return acc.value();
}

// After the first barrier of a launch that split the FP64 field: every CTA has read the flag,
// so the team's rank 0 marks the triple-float field current (it persists across launches:
// the FP64 field is only its rounding, rewritten at the end of every launch).
__device__ __forceinline__ void mark_split(const CaseDev& cs, const Team& tm, bool& convert) {
  if (convert && tm.rank == 0 && threadIdx.x == 0) *reinterpret_cast<volatile int32_t*>(cs.flags) = 1;
  convert = false;
}

// The FP64 field from the triple-float one (end of the launch; each CTA its own cells), with
// the last solve's correction added to the triple-float field first when it is not yet.
template <int B>
__device__ __noinline__ void pass_store_x(const CaseDev& cs, int c0, int c1, bool fold) {
  float2* __restrict__ x2 = cs.x2;
  float* __restrict__ xl = cs.xlo;
  double* __restrict__ x = cs.x;
  for (int c = c0 + (int)threadIdx.x; c < c1; c += B) {
    tf v = ld_tf(x2, xl, c);
    if (fold) {  // the triple-float field carries over to the next launch: keep it current
      v = tf_add_df(v, ld_df(cs.e2 + c));
      st_tf(x2, xl, c, v);
    }
    x[c] = tf_to_double(v);
  }
}

// Boundary conductance, source and flux g_b (T_b - x_c) of row c (fixedValue faces;
// zeroGradient adds nothing), in FP64 with the case scale, in ascending face order.
__device__ __forceinline__ void row_boundary_df(const CaseDev& cs, int c, tf xc, df& gsum, df& ssum, df& flux) {
  const int b0 = __ldg(cs.b_start + c), b1 = __ldg(cs.b_start + c + 1);
  gsum = mkdf(0.0f, 0.0f);
  ssum = mkdf(0.0f, 0.0f);
  flux = mkdf(0.0f, 0.0f);
  if (b0 == b1) return;
  const double x = tf_to_double(xc);
  double g = 0.0, s = 0.0, fl = 0.0;
  for (int k = b0; k < b1; ++k) {
    const int bf = LFM_IDX(__ldg(cs.b_face + k), cs.NB, 0, kChkBFace);
    if (__ldg(cs.btype + bf) == LFM_FIXED_VALUE) {
      const double gb = __ldg(cs.bDT + bf) * __ldg(cs.bmagSf + bf) * __ldg(cs.bdelta + bf) * cs.df_scale;
      const double tb = __ldg(cs.bval + bf);
      g += gb;
      s += gb * tb;
      fl += gb * (tb - x);
    }
  }
  gsum = df_from_double(g);
  ssum = df_from_double(s);
  flux = df_from_double(fl);
}

// ---- general geometry ----------------------------------------------------------------
// G: the Gauss linear gradient of the field over [c0, c1) into grad2, in difference form
//   G_c = sum_k gE_k (T_k - T_c) + sum_fixedValue (bSf / V)(T_b - T_c) + gZ T_c
// (equal to the operator form gD T_c + gH + sum_k gE_k T_k; see CaseDev): a weighted sum of
// T values that nearly cancel would carry their rounding, ~2^-48 |T| / h, into the explicit
// correction; differences formed exactly from the triple-float field do not. The boundary
// terms (boundary cells only) are FP64; gZ T_c (gZ is zero up to the geometry's rounding) df64.
template <int B, int W>
__device__ __noinline__ void pass_grad_df(const CaseDev& cs, int c0, int c1) {
  const float2* __restrict__ x2 = cs.x2;
  const float* __restrict__ xl = cs.xlo;
  const size_t N = (size_t)cs.N;
  const int ns = W > 0 ? W : cs.W;
  const size_t WN = (size_t)ns * N;
  for (int c = c0 + (int)threadIdx.x; c < c1; c += B) {
    const tf xc = ld_tf(x2, xl, c);
    df g0 = mkdf(0.0f, 0.0f), g1 = g0, g2 = g0;
#pragma unroll
    for (int k = 0; k < (W > 0 ? W : kMaxSlots); ++k) {
      if (W == 0 && k >= ns) break;
      const size_t at = (size_t)k * N + c;
      const df d = tf_diff(ld_tf(x2, xl, LFM_IDX(__ldg(cs.slot_other + at), cs.N, c, kChkSlotCellDf)), xc);
      g0 = df_fma(ldg_df(cs.gE2 + at), d, g0);
      g1 = df_fma(ldg_df(cs.gE2 + WN + at), d, g1);
      g2 = df_fma(ldg_df(cs.gE2 + 2 * WN + at), d, g2);
    }
    const df xcd = tf_to_df(xc);
    g0 = df_fma(ldg_df(cs.gZ + c), xcd, g0);
    g1 = df_fma(ldg_df(cs.gZ + N + c), xcd, g1);
    g2 = df_fma(ldg_df(cs.gZ + 2 * N + c), xcd, g2);
    const int k0 = __ldg(cs.b_start + c), k1 = __ldg(cs.b_start + c + 1);
    if (k0 != k1) {  // boundary cells: the fixedValue faces' terms in FP64
      const double xd = tf_to_double(xc), rv = 1.0 / cs.V[c];
      double b0 = 0.0, b1 = 0.0, b2 = 0.0;
      for (int k = k0; k < k1; ++k) {
        const int bf = LFM_IDX(__ldg(cs.b_face + k), cs.NB, 0, kChkBFace);
        if (__ldg(cs.btype + bf) == LFM_FIXED_VALUE) {
          const double dT = (__ldg(cs.bval + bf) - xd) * rv;
          b0 = fma(cs.bSf[3 * (size_t)bf], dT, b0);
          b1 = fma(cs.bSf[3 * (size_t)bf + 1], dT, b1);
          b2 = fma(cs.bSf[3 * (size_t)bf + 2], dT, b2);
        }
      }
      g0 = df_add(g0, df_from_double(b0));
      g1 = df_add(g1, df_from_double(b1));
      g2 = df_add(g2, df_from_double(b2));
    }
    st_df(cs.grad2 + c, g0);
    st_df(cs.grad2 + N + c, g1);
    st_df(cs.grad2 + 2 * N + c, g2);
  }
}

// The explicit non-orthogonal correction of row c (scaled with the system): the sum over the
// cell's faces of the correction flux, through the weights cK, cL of the gradient.
template <int W>
__device__ __forceinline__ df op_corr_df(const CaseDev& cs, int c) {
  const size_t N = (size_t)cs.N;
  const int ns = W > 0 ? W : cs.W;
  const size_t WN = (size_t)ns * N;
  const float2* __restrict__ G = cs.grad2;
  df v = df_mul(ldg_df(cs.cK2 + c), ld_df(G + c));
  v = df_fma(ldg_df(cs.cK2 + N + c), ld_df(G + N + c), v);
  v = df_fma(ldg_df(cs.cK2 + 2 * N + c), ld_df(G + 2 * N + c), v);
#pragma unroll
  for (int k = 0; k < (W > 0 ? W : kMaxSlots); ++k) {
    if (W == 0 && k >= ns) break;
    const size_t at = (size_t)k * N + c;
    const int o = LFM_IDX(__ldg(cs.slot_other + at), cs.N, c, kChkSlotCellDf);
    v = df_fma(ldg_df(cs.cL2 + at), ld_df(G + o), v);
    v = df_fma(ldg_df(cs.cL2 + WN + at), ld_df(G + N + o), v);
    v = df_fma(ldg_df(cs.cL2 + 2 * WN + at), ld_df(G + 2 * N + o), v);
  }
  return v;
}

// L2 prefetch of what a row pass loads for row c before its gathers: the slot indices and
// conductances, the field value and V/dt. Issued one trip ahead (c + B), it shortens the
// dependent chain index -> neighbour value of the next row (row pass 0.32 -> 0.30 ms per
// step on the 200^3 graded box).
template <int W>
__device__ __forceinline__ void prefetch_row_df(const CaseDev& cs, int c) {
  const size_t N = (size_t)cs.N;
  const int ns = W > 0 ? W : cs.W;
  for (int k = 0; k < (W > 0 ? W : kMaxSlots); ++k) {
    if (W == 0 && k >= ns) break;
    prefetch_l2(cs.slot_other + (size_t)k * N + c);
    prefetch_l2(cs.g2 + (size_t)k * N + c);
  }
  prefetch_l2(cs.x2 + c);
  prefetch_l2(cs.xlo + c);
  prefetch_l2(cs.vdt2 + c);
}

// R: rows of the matrix and, from the same loaded row, the initial residual, normFactor
// terms, sum|r| and rho; p = w. kSrc: correctors (ddt source from x_old) or volumetric
// sources present.
// The residual is evaluated in flux form,
//   r_c = sum_k g_k (x_other(k) - x_c) + sum_b g_b (T_b - x_c) + V/dt (x_old,c - x_c)
//         + V Su_c + V Sp_c x_c,
// which equals b - A x term by term. Formed as b - A x, r would be the small difference of
// two values of order V/dt T and carry their rounding error, ~2^-48 |b|, amplified by
// |b| / |r| (about 1e6 for a time step that changes T by one part in a million); the
// differences of nearby values here are almost exact, so r keeps the format's relative
// accuracy. A x for the normFactor terms is then b - r.
template <int B, int W, bool kSrc>
__device__ __noinline__ Sums3 pass_rows_init_df(const CaseDev& cs, int c0, int c1, double xRef) {
  const float2* __restrict__ x2 = cs.x2;
  const float* __restrict__ xl = cs.xlo;
  const float2* __restrict__ g2 = cs.g2;
  float2* __restrict__ r2 = reinterpret_cast<float2*>(cs.r);
  float2* __restrict__ p2 = reinterpret_cast<float2*>(cs.p);
  const size_t N = (size_t)cs.N;
  const df xr = df_from_scalar(xRef);
  DfAcc a_nf, a_r, a_rho;
  for (int c = c0 + (int)threadIdx.x; c < c1; c += B) {
    if (c + B < c1) prefetch_row_df<W>(cs, c + B);
    const tf xc = ld_tf(x2, xl, c);
    df d, flux;
    if constexpr (W > 0) {
      int o[W];
      df g[W];
#pragma unroll
      for (int k = 0; k < W; ++k) {
        o[k] = LFM_IDX(__ldg(cs.slot_other + (size_t)k * N + c), cs.N, c, kChkSlotCellDf);
        g[k] = ldg_df(g2 + (size_t)k * N + c);
      }
      tf xo_[W];
#pragma unroll
      for (int k = 0; k < W; ++k) xo_[k] = ld_tf(x2, xl, o[k]);
      d = g[0];
#pragma unroll
      for (int k = 1; k < W; ++k) d = df_add(d, g[k]);  // padding slots hold 0
      flux = df_mul(g[0], tf_diff(xo_[0], xc));
#pragma unroll
      for (int k = 1; k < W; ++k) flux = df_fma(g[k], tf_diff(xo_[k], xc), flux);
    } else {
      d = mkdf(0.0f, 0.0f);
      flux = mkdf(0.0f, 0.0f);
      for (int k = 0; k < cs.W; ++k) {
        const size_t at = (size_t)k * N + c;
        const df gk = ldg_df(g2 + at);
        d = df_add(d, gk);
        flux = df_fma(gk, tf_diff(ld_tf(x2, xl, LFM_IDX(__ldg(cs.slot_other + at), cs.N, c, kChkSlotCellDf)), xc), flux);
      }
    }
    df gb, sb, fb;
    row_boundary_df(cs, c, xc, gb, sb, fb);
    const df vdt = ldg_df(cs.vdt2 + c);
    const df xcd = tf_to_df(xc);
    const bool has_old = kSrc && cs.n_corr > 0;
    const tf xo = has_old ? ld_tf(reinterpret_cast<const float2*>(cs.x_old), cs.xolo, c) : xc;
    d = df_add(df_add(d, gb), vdt);
    df src = df_fma(vdt, has_old ? tf_to_df(xo) : xcd, sb);
    df sa = df_add(vdt, gb);
    df rc = df_add(flux, fb);
    if (has_old) rc = df_fma(vdt, tf_diff(xo, xc), rc);
    if (kSrc && (cs.vSp || cs.vSu)) {
      // the volumetric source V Su + V Sp T of the row's residual, in FP64 (proportional to T)
      const double sp = cs.vSp ? cs.vSp[c] * cs.df_scale : 0.0;
      const double su = cs.vSu ? cs.vSu[c] * cs.df_scale : 0.0;
      const df vsp = df_from_double(sp);
      d = df_sub(d, vsp);
      sa = df_sub(sa, vsp);
      src = df_add(src, df_from_double(su));
      rc = df_add(rc, df_from_double(fma(sp, tf_to_double(xc), su)));
    }
    if (kSrc && cs.Sf) {  // the explicit non-orthogonal correction joins the source
      const df corr = op_corr_df<W>(cs, c);
      src = df_add(src, corr);
      rc = df_add(rc, corr);
    }
    const df ax = df_sub(src, rc);
    const df rd = df_rcp(d);
    const df sx = df_mul(sa, xr);
    a_nf.add(df_abs(df_sub(ax, sx)));
    a_nf.add(df_abs(df_sub(src, sx)));
    a_r.add(df_abs(rc));
    const df wc = df_mul(rd, rc);
    a_rho.add(df_mul(wc, rc));
    st_df(cs.diag2 + c, d);
    st_df(cs.rD2 + c, rd);
    st_df(r2 + c, rc);
    st_df(p2 + c, wc);
  }
  return Sums3{a_nf.value(), a_r.value(), a_rho.value()};
}

// Rows c and c2 of A v, all loads of both rows issued before any is used; the matrix arrays
// with evict-first (streaming) loads, so that they do not displace the gathered vector.
template <int W>
__device__ __forceinline__ void rows2_df(const CaseDev& cs, int c, int c2, const float2* __restrict__ v, df& y,
                                         df& y2, df& vc, df& vc2) {
  const size_t N = (size_t)cs.N;
  const float2* __restrict__ g2 = cs.g2;
  vc = ld_df(v + c);
  vc2 = ld_df(v + c2);
  const float2 dd1 = __ldcs(cs.diag2 + c), dd2 = __ldcs(cs.diag2 + c2);
  df acc = df_mul(df{dd1.x, dd1.y}, vc), acc2 = df_mul(df{dd2.x, dd2.y}, vc2);
  if constexpr (W > 0) {
    int o[W], o2[W];
    df g[W], h[W];
#pragma unroll
    for (int k = 0; k < W; ++k) {
      o[k] = LFM_IDX(__ldcs(cs.slot_other + (size_t)k * N + c), cs.N, c, kChkSlotCellDf);
      o2[k] = LFM_IDX(__ldcs(cs.slot_other + (size_t)k * N + c2), cs.N, c2, kChkSlotCellDf);
      const float2 a = __ldcs(g2 + (size_t)k * N + c), b = __ldcs(g2 + (size_t)k * N + c2);
      g[k] = df{a.x, a.y};
      h[k] = df{b.x, b.y};
    }
#pragma unroll
    for (int k = 0; k < W; ++k) {
      acc = df_fma(df_neg(g[k]), ld_df(v + o[k]), acc);
      acc2 = df_fma(df_neg(h[k]), ld_df(v + o2[k]), acc2);
    }
  } else {
    for (int k = 0; k < cs.W; ++k) {
      const size_t at = (size_t)k * N;
      acc = df_fma(df_neg(ldg_df(g2 + at + c)), ld_df(v + LFM_IDX(__ldg(cs.slot_other + at + c), cs.N, c, kChkSlotCellDf)), acc);
      acc2 = df_fma(df_neg(ldg_df(g2 + at + c2)), ld_df(v + LFM_IDX(__ldg(cs.slot_other + at + c2), cs.N, c2, kChkSlotCellDf)), acc2);
    }
  }
  y = acc;
  y2 = acc2;
}

template <int W>
__device__ __forceinline__ df row1_df(const CaseDev& cs, int c, const float2* __restrict__ v, df& vc) {
  const size_t N = (size_t)cs.N;
  const int ns = W > 0 ? W : cs.W;
  vc = ld_df(v + c);
  df acc = df_mul(ld_df(cs.diag2 + c), vc);
#pragma unroll
  for (int k = 0; k < (W > 0 ? W : kMaxSlots); ++k) {
    if (W == 0 && k >= ns) break;
    const size_t at = (size_t)k * N + c;
    acc = df_fma(df_neg(ldg_df(cs.g2 + at)), ld_df(v + LFM_IDX(__ldg(cs.slot_other + at), cs.N, c, kChkSlotCellDf)), acc);
  }
  return acc;
}

// P: p = w + beta p.
template <int B>
__device__ __forceinline__ void pass_direction_df(int c0, int c1, df beta, float2* __restrict__ p,
                                                  const float2* __restrict__ w) {
  int c = c0 + (int)threadIdx.x;
  for (; c + B < c1; c += 2 * B) {
    pf_next<B>(p, c, c1);
    pf_next<B>(w, c, c1);
    const df p1 = ld_df(p + c), p2 = ld_df(p + c + B), w1 = ld_df(w + c), w2 = ld_df(w + c + B);
    st_df(p + c, df_fma(beta, p1, w1));
    st_df(p + c + B, df_fma(beta, p2, w2));
  }
  if (c < c1) st_df(p + c, df_fma(beta, ld_df(p + c), ld_df(w + c)));
}

// M: q = A p; returns this thread's share of p.q.
template <int B, int W>
__device__ __forceinline__ double pass_amul_dot_df(const CaseDev& cs, int c0, int c1, const float2* __restrict__ p,
                                                   float2* __restrict__ q) {
  DfAcc s;
  int c = c0 + (int)threadIdx.x;
  for (; c + B < c1; c += 2 * B) {
    df y1, y2, pc1, pc2;
    rows2_df<W>(cs, c, c + B, p, y1, y2, pc1, pc2);
    st_df(q + c, y1);
    st_df(q + c + B, y2);
    s.add(df_mul(y1, pc1));
    s.add(df_mul(y2, pc2));
  }
  if (c < c1) {
    df pc;
    const df y = row1_df<W>(cs, c, p, pc);
    st_df(q + c, y);
    s.add(df_mul(y, pc));
  }
  return s.value();
}

// U: e += alpha p (first iteration of a solve: e = alpha p), r -= alpha q, w = rD r; returns
// this thread's sum|r| and w.r. e, the solve's correction to the field, is added to the
// triple-float field once per solve (pass_sum_df, pass_store_x), so an iteration moves 8
// bytes of field state per cell instead of reading and writing the field's 12.
template <int B>
__device__ __forceinline__ double2 pass_update_df(int c0, int c1, df alpha, float2* __restrict__ e, bool first,
                                                  float2* __restrict__ r, float2* __restrict__ w,
                                                  const float2* __restrict__ p, const float2* __restrict__ q,
                                                  const float2* __restrict__ rD) {
  DfAcc sa, sr;
  const df nalpha = df_neg(alpha);
  int c = c0 + (int)threadIdx.x;
  for (; c + B < c1; c += 2 * B) {
    const int k = c + B;
    const df pa = ld_df(p + c), pb = ld_df(p + k), qa = ld_df(q + c), qb = ld_df(q + k);
    const df ra = ld_df(r + c), rb = ld_df(r + k);
    const df da = ld_df(rD + c), db = ld_df(rD + k);
    const df rna = df_fma(nalpha, qa, ra), rnb = df_fma(nalpha, qb, rb);
    const df wa = df_mul(da, rna), wb = df_mul(db, rnb);
    if (first) {
      st_df(e + c, df_mul(alpha, pa));
      st_df(e + k, df_mul(alpha, pb));
    } else {
      const df ea = ld_df(e + c), eb = ld_df(e + k);
      st_df(e + c, df_fma(alpha, pa, ea));
      st_df(e + k, df_fma(alpha, pb, eb));
    }
    st_df(r + c, rna);
    st_df(r + k, rnb);
    st_df(w + c, wa);
    st_df(w + k, wb);
    sa.add(df_abs(rna));
    sa.add(df_abs(rnb));
    sr.add(df_mul(wa, rna));
    sr.add(df_mul(wb, rnb));
  }
  if (c < c1) {
    const df rn = df_fma(nalpha, ld_df(q + c), ld_df(r + c));
    const df wn = df_mul(ld_df(rD + c), rn);
    const df pc = ld_df(p + c);
    st_df(e + c, first ? df_mul(alpha, pc) : df_fma(alpha, pc, ld_df(e + c)));
    st_df(r + c, rn);
    st_df(w + c, wn);
    sa.add(df_abs(rn));
    sr.add(df_mul(wn, rn));
  }
  return make_double2(sa.value(), sr.value());
}

// The steps of one launch. Returns false when a barrier failed (the caller leaves).
// `pending` tracks whether e holds a correction not yet added to the field (the same in every
// CTA: it follows the team-wide iteration counts).
template <int B, int W, bool kGeom>
__device__ bool steps_df64(const CaseDev& cs, const CaseDev& cref, const Team& tm, int n_steps, TeamShared& sh,
                           int stats_base, int c0, int c1, bool& pending) {
  const int tid = threadIdx.x;
  float2* __restrict__ e = cs.e2;
  float2* __restrict__ r = reinterpret_cast<float2*>(cs.r);
  float2* __restrict__ w = reinterpret_cast<float2*>(cs.w);
  float2* __restrict__ p = reinterpret_cast<float2*>(cs.p);
  float2* __restrict__ q = reinterpret_cast<float2*>(cs.q);
  const float2* __restrict__ rD = cs.rD2;
  const double inv_scale = 1.0 / cs.df_scale;  // a power of two: exact

  PhaseClock clk(cs, tm);
  const bool src_mode = cs.n_corr > 0 || cs.vSu != nullptr || cs.vSp != nullptr || (kGeom && cs.Sf != nullptr);
  bool convert = ld_volatile_i32(cs.flags) == 0;  // read by every CTA before the first barrier
  for (int step = 0; step < n_steps; ++step) {
    int iters_tot = 0, solves = 0, status = 0;
    double nf0 = 0.0, init0 = 0.0, res = 0.0;
    bool conv = false;
    for (int pass = 0; pass <= cs.n_corr; ++pass) {
      // ---- S: sum of x (first pass of the launch: split the FP64 field; otherwise the last
      //      solve's correction is added first) ---------------------------------------------
      double v[1] = {pass_sum_df<B>(cref, c0, c1, convert, pending, pass == 0 && cs.n_corr > 0)};
      pending = false;
      if (!team_allreduce<1>(tm, v, sh)) return false;
      mark_split(cs, tm, convert);
      if constexpr (kGeom) {
        if (cs.Sf) {  // ---- G: the gradient of the (folded) field, for the correction --------
          pass_grad_df<B, W>(cref, c0, c1);
          if (!team_barrier(tm, sh)) return false;
        }
      }
      clk.lap(kPhAssembly);
      // ---- R: rows, initial residual, normFactor, first direction ----------------------
      const double xRef = v[0] / (double)cs.N;
      const Sums3 ui = src_mode ? pass_rows_init_df<B, W, true>(cref, c0, c1, xRef)
                                : pass_rows_init_df<B, W, false>(cref, c0, c1, xRef);
      double u[3] = {ui.a, ui.b, ui.c};
      if (!team_allreduce<3>(tm, u, sh)) return false;
      clk.lap(kPhInit);
      const double nf = u[0] + kSmall * cs.df_scale;
      const double init_res = u[1] / nf;
      res = init_res;
      double rho = u[2], beta = 0.0;
      int iters = 0;
      conv = converged(res, init_res, cs.tol, cs.rel_tol);
      if (cs.min_iter > 0 || !conv) {
        for (;;) {
          if (iters > 0) {
            pass_direction_df<B>(c0, c1, df_from_scalar(beta), p, w);
            if (!team_barrier(tm, sh)) return false;
            clk.lap(kPhP);
          }
          double s1[1] = {pass_amul_dot_df<B, W>(cs, c0, c1, p, q)};
          if (!team_allreduce<1>(tm, s1, sh)) return false;
          clk.lap(kPhM);
          const double sigma = s1[0];
          if (fabs(sigma) / nf < kVSmall) {
            status = LFM_ESINGULAR;
            break;
          }
          const double alpha = rho / sigma;
          const double2 su = pass_update_df<B>(c0, c1, df_from_scalar(alpha), e, iters == 0, r, w, p, q, rD);
          pending = true;
          double s2[2] = {su.x, su.y};
          if (!team_allreduce<2>(tm, s2, sh)) return false;
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
        nf0 = nf * inv_scale;
        init0 = init_res;
      }
      iters_tot += iters;
      solves += iters > 0 ? 1 : 0;
      if (status != 0) break;
    }
    write_stats(cs, tm, stats_base + step, iters_tot, conv ? 1 : 0, solves, status, init0, res, nf0);
    if (status != 0) {
      if (tm.rank == 0 && tid == 0) set_status(cs.sync, status);
      return true;
    }
  }
  return true;
}

// kGeom: the kernel serves general geometry (the gradient phase is compiled in).
template <int B, int W, bool kGeom = false>
__device__ void run_steps_df64(const CaseDev& cs, const CaseDev& cref, const Team& tm, int n_steps, TeamShared& sh,
                               int stats_base = 0) {
  if (n_steps <= 0) return;
  int c0, c1;
  cta_range(cs.N, tm.size, tm.rank, c0, c1);
  bool pending = false;
  steps_df64<B, W, kGeom>(cs, cref, tm, n_steps, sh, stats_base, c0, c1, pending);
  // the field and the correction of the CTA's own cells are written by this CTA only, so the
  // FP64 field can be written back without another barrier, also after an early exit.
  pass_store_x<B>(cref, c0, c1, pending);
}

}  // namespace
}  // namespace lfm

// lfm_solve_mixed_df.cuh -- the mixed form's steps with df64 outer passes, shared by the
// single-case kernel (lfm_step.cu) and the batched kernel (lfm_batch.cu).
//
// The mixed form's defect correction (FP32 inner CG on A dx = r, FP64-class outer residual;
// lfm_solve.cuh) with its outer passes in the df64 machinery of lfm_solve_df.cuh: the field
// as a triple-float, the true residual in flux form, the correction x += dx on the FP32 pipe.
// The inner solve works in the unscaled units of the FP32 slot coefficients: the outer passes
// hand it r / s, diag / s and s / diag (s the case's power-of-two scale, exact), and the
// scalars it tests are unscaled too.
//
// Per step (phases separated by team barriers):
//   S   sum of x (xRef); x kept as the step's starting field x_old
//   T0  rows of the matrix (FP32 copies of diag and 1/diag for the inner solve), the true
//       residual r = b - A x, normFactor, and the seed of the inner solve
//   sweep: inner CG (P, M, U on FP32 vectors; M with its matrix rows bulk-copied into shared
//          memory where the launch provides it) on A dx = r; C  x += dx, sum of x;
//          then the true residual after the correction: T1, or V (below); another sweep
//          while it is not converged
// V (steps without volumetric sources or non-orthogonal correctors): one pass over the rows
// gives the verification residual of the step, r_v = b - A x, and the next step's assembly
// and first residual. Their flux forms share every face term:
//   r_v   = sum_k g_k (x_other(k) - x_c) + sum_b g_b (T_b - x_c) + V/dt (x_old,c - x_c)
//   r'    = sum_k g_k (x_other(k) - x_c) + sum_b g_b (T_b - x_c)
// (the next step starts from this x, so its ddt term vanishes), and xRef of the next step is
// the sum of x that C returned. The next step then starts at its inner solve: S and T0 are
// not repeated, and its first C keeps x_old. Every value is formed by the same operations in
// the same order as S and T0 would form it, so the results are those of the unfused sequence
// bit for bit. When the verification asks for another sweep, T1 re-seeds the inner solve
// from r_v.
#pragma once

#include <cuda_runtime.h>

#include "lfm_device.cuh"
#include "lfm_df64.cuh"
#include "lfm_internal.h"
#include "lfm_solve.cuh"
#include "lfm_solve_df.cuh"

namespace lfm {
namespace {

// Row c's face part in flux form over the slots (slot order): flux = sum_k g_k (x_other(k) -
// x_c) and, with kDiag, the sum d of the slot conductances (the diagonal's face part).
template <int W, bool kDiag>
__device__ __forceinline__ void row_flux_df(const CaseDev& cs, int c, const tf& xc, df& d, df& flux) {
  const float2* __restrict__ x2 = cs.x2;
  const float* __restrict__ xl = cs.xlo;
  const float2* __restrict__ g2 = cs.g2;
  const size_t N = (size_t)cs.N;
  if constexpr (W > 0) {
    int o[W];
    df g[W];
#pragma unroll
    for (int k = 0; k < W; ++k) {
      o[k] = LFM_IDX(__ldg(cs.slot_other + (size_t)k * N + c), cs.N, c, kChkSlotCellDf);
      g[k] = ldg_df(g2 + (size_t)k * N + c);
    }
    tf xo[W];
#pragma unroll
    for (int k = 0; k < W; ++k) xo[k] = ld_tf(x2, xl, o[k]);
    if constexpr (kDiag) {
      d = g[0];
#pragma unroll
      for (int k = 1; k < W; ++k) d = df_add(d, g[k]);  // padding slots hold 0
    }
    flux = df_mul(g[0], tf_diff(xo[0], xc));
#pragma unroll
    for (int k = 1; k < W; ++k) flux = df_fma(g[k], tf_diff(xo[k], xc), flux);
  } else {
    d = mkdf(0.0f, 0.0f);
    flux = mkdf(0.0f, 0.0f);
    for (int k = 0; k < cs.W; ++k) {
      const size_t at = (size_t)k * N + c;
      const df gk = ldg_df(g2 + at);
      if constexpr (kDiag) d = df_add(d, gk);
      flux = df_fma(gk, tf_diff(ld_tf(x2, xl, LFM_IDX(__ldg(cs.slot_other + at), cs.N, c, kChkSlotCellDf)), xc), flux);
    }
  }
}

// The rest of a step's first row pass once the row is assembled (diag d, source src, row sum
// sa, residual rc; all scaled): A x = src - rc and the normFactor terms against xRef (xr),
// sum|r|, and the inner solve's seed r32 = r / s, w32 = rD32 r32, p32 = w32 (dx32 starts at zero
// implicitly: the solve's first update writes it),
// rho = w32.r32 (FP32 pairs), with the FP32 copies of diag / s and s / diag.
__device__ __forceinline__ void seed_row_df(const CaseDev& cs, int c, df d, df src, df sa, df rc, df xr, float s32,
                                            float inv_s32, DfAcc& a_nf, DfAcc& a_r, Acc2f& a_rho) {
  const df ax = df_sub(src, rc);
  const df rd = df_rcp(d);
  const df sx = df_mul(sa, xr);
  a_nf.add(df_abs(df_sub(ax, sx)));
  a_nf.add(df_abs(df_sub(src, sx)));
  a_r.add(df_abs(rc));
  const float rd32 = __fmul_rn(rd.hi, s32);
  const float r32 = __fmul_rn(rc.hi, inv_s32);
  const float w32 = __fmul_rn(rd32, r32);
  a_rho.add_prod(w32, r32);
  cs.diag32[c] = __fmul_rn(d.hi, inv_s32);
  cs.rD32[c] = rd32;
  cs.r32[c] = r32;
  cs.w32[c] = w32;
  cs.p32[c] = w32;
}

// T0: rows of the matrix, the true residual (flux form), normFactor terms, sum|r| (scaled;
// the caller unscales) and the seed of the inner solve. kSrc: correctors (ddt source from
// x_old) or volumetric sources present.
template <int B, int W, bool kSrc>
__device__ __noinline__ Sums3 pass_rows_init_mixed_df(const CaseDev& cs, int c0, int c1, double xRef, float s32,
                                                      float inv_s32) {
  const df xr = df_from_scalar(xRef);
  DfAcc a_nf, a_r;
  Acc2f a_rho;
  for (int c = c0 + (int)threadIdx.x; c < c1; c += B) {
    if (c + B < c1) prefetch_row_df<W>(cs, c + B);
    const tf xc = ld_tf(cs.x2, cs.xlo, c);
    df d, flux;
    row_flux_df<W, true>(cs, c, xc, d, flux);
    df gb, sb, fb;
    row_boundary_df(cs, c, xc, gb, sb, fb);
    const df vdt = ldg_df(cs.vdt2 + c);
    const bool has_old = kSrc && cs.n_corr > 0;
    const tf xo = has_old ? ld_tf(reinterpret_cast<const float2*>(cs.x_old), cs.xolo, c) : xc;
    d = df_add(df_add(d, gb), vdt);
    df src = df_fma(vdt, tf_to_df(xo), sb);
    df sa = df_add(vdt, gb);
    df rc = df_add(flux, fb);
    if (has_old) rc = df_fma(vdt, tf_diff(xo, xc), rc);
    if (kSrc && (cs.vSp || cs.vSu)) {
      const double sp = cs.vSp ? cs.vSp[c] * cs.df_scale : 0.0;
      const double su = cs.vSu ? cs.vSu[c] * cs.df_scale : 0.0;
      const df vsp = df_from_double(sp);
      d = df_sub(d, vsp);
      sa = df_sub(sa, vsp);
      src = df_add(src, df_from_double(su));
      rc = df_add(rc, df_from_double(fma(sp, tf_to_double(xc), su)));
    }
    seed_row_df(cs, c, d, src, sa, rc, xr, s32, inv_s32, a_nf, a_r, a_rho);
  }
  return Sums3{a_nf.value(), a_r.value(), a_rho.value()};
}

// T1: the true residual after a correction, in flux form (x differs from the step's starting
// field x_old now); sum|r| (scaled) and the seed of the next inner solve as in T0.
template <int B, int W, bool kSrc>
__device__ __noinline__ double2 pass_true_residual_df(const CaseDev& cs, int c0, int c1, float inv_s32) {
  DfAcc a_r;
  Acc2f a_rho;
  for (int c = c0 + (int)threadIdx.x; c < c1; c += B) {
    const tf xc = ld_tf(cs.x2, cs.xlo, c);
    df d, flux;
    row_flux_df<W, false>(cs, c, xc, d, flux);
    df gb, sb, fb;
    row_boundary_df(cs, c, xc, gb, sb, fb);
    const tf xo = ld_tf(reinterpret_cast<const float2*>(cs.x_old), cs.xolo, c);
    df rc = df_fma(ldg_df(cs.vdt2 + c), tf_diff(xo, xc), df_add(flux, fb));
    if (kSrc && (cs.vSp || cs.vSu)) {
      const double sp = cs.vSp ? cs.vSp[c] * cs.df_scale : 0.0;
      const double su = cs.vSu ? cs.vSu[c] * cs.df_scale : 0.0;
      rc = df_add(rc, df_from_double(fma(sp, tf_to_double(xc), su)));
    }
    a_r.add(df_abs(rc));
    const float r32 = __fmul_rn(rc.hi, inv_s32);
    const float w32 = __fmul_rn(cs.rD32[c], r32);
    a_rho.add_prod(w32, r32);
    cs.r32[c] = r32;
    cs.w32[c] = w32;
    cs.p32[c] = w32;
  }
  return make_double2(a_r.value(), a_rho.value());
}

// Four partial sums of a pass, per thread.
struct Sums4 {
  double a, b, c, d;
};

// V: the step's verification residual and the next step's T0 in one pass over the rows (no
// sources, no correctors; see the head of this file). xRef_next: mean of the corrected x.
// Returns sum|r_v| (scaled), then the next step's normFactor sum, sum|r'| and rho.
template <int B, int W>
__device__ __noinline__ Sums4 pass_verify_next_df(const CaseDev& cs, int c0, int c1, double xRef_next, float s32,
                                                    float inv_s32) {
  const df xr = df_from_scalar(xRef_next);
  DfAcc a_v, a_nf, a_r;
  Acc2f a_rho;
  for (int c = c0 + (int)threadIdx.x; c < c1; c += B) {
    if (c + B < c1) {
      prefetch_row_df<W>(cs, c + B);
      // and the next row's per-cell values only this pass reads
      prefetch_l2(cs.x_old + c + B);
      prefetch_l2(cs.xolo + c + B);
      prefetch_l2(cs.b_start + c + B);
    }
    const tf xc = ld_tf(cs.x2, cs.xlo, c);
    df d, flux;
    row_flux_df<W, true>(cs, c, xc, d, flux);
    df gb, sb, fb;
    row_boundary_df(cs, c, xc, gb, sb, fb);
    const df vdt = ldg_df(cs.vdt2 + c);
    const tf xo = ld_tf(reinterpret_cast<const float2*>(cs.x_old), cs.xolo, c);
    const df rn = df_add(flux, fb);  // the next step's first residual
    a_v.add(df_abs(df_fma(vdt, tf_diff(xo, xc), rn)));
    d = df_add(df_add(d, gb), vdt);
    seed_row_df(cs, c, d, df_fma(vdt, tf_to_df(xc), sb), df_add(vdt, gb), rn, xr, s32, inv_s32, a_nf, a_r, a_rho);
  }
  return Sums4{a_v.value(), a_nf.value(), a_r.value(), a_rho.value()};
}

// C: x += dx (the triple-float field and the FP32 correction of the inner solve). save_old:
// keep x before the correction as the step's starting field (the first correction of a step
// that began without S). Returns this thread's sum of the corrected x, formed as S forms it.
// Two cells per loop trip (c, c + B), all their loads issued first and the next trip's
// prefetched into L2; the sum is taken in the same order as one cell per trip.
template <int B>
__device__ __noinline__ double pass_correct_df(const CaseDev& cs, int c0, int c1, bool save_old) {
  float2* __restrict__ x2 = cs.x2;
  float* __restrict__ xl = cs.xlo;
  const float* __restrict__ dx = cs.dx32;
  float2* __restrict__ xo2 = reinterpret_cast<float2*>(cs.x_old);
  DfAcc acc;
  int c = c0 + (int)threadIdx.x;
  for (; c + B < c1; c += 2 * B) {
    pf_next<B>(x2, c, c1);
    pf_next<B>(xl, c, c1);
    pf_next<B>(dx, c, c1);
    const int e = c + B;
    tf a = ld_tf(x2, xl, c), b = ld_tf(x2, xl, e);
    const float da = dx[c], db = dx[e];
    if (save_old) {
      st_tf(xo2, cs.xolo, c, a);
      st_tf(xo2, cs.xolo, e, b);
    }
    a = tf_add_df(a, mkdf(da, 0.0f));
    b = tf_add_df(b, mkdf(db, 0.0f));
    st_tf(x2, xl, c, a);
    st_tf(x2, xl, e, b);
    acc.add(tf_to_df(a));
    acc.add(tf_to_df(b));
  }
  if (c < c1) {
    tf v = ld_tf(x2, xl, c);
    if (save_old) st_tf(xo2, cs.xolo, c, v);
    v = tf_add_df(v, mkdf(dx[c], 0.0f));
    st_tf(x2, xl, c, v);
    acc.add(tf_to_df(v));
  }
  return acc.value();
}

// Whether the mixed form of this case runs its outer passes in df64: the df64 arrays are
// present, the mesh is orthogonal and the scale is an FP32 power of two.
__device__ __forceinline__ bool mixed_uses_df(const CaseDev& cs) {
  return cs.x2 != nullptr && cs.Sf == nullptr && cs.df_scale >= 0x1p-100 && cs.df_scale <= 0x1p100;
}

template <int B, int W>
__device__ bool steps_mixed_df(const CaseDev& cs, const CaseDev& cref, const Team& tm, int n_steps, TeamShared& sh,
                               int stats_base, int c0, int c1) {
  const int tid = threadIdx.x;
  float* __restrict__ dx = cs.dx32;
  float* __restrict__ r = cs.r32;
  float* __restrict__ w = cs.w32;
  float* __restrict__ p = cs.p32;
  float* __restrict__ q = cs.q32;
  const float* __restrict__ rD = cs.rD32;
  const double inv_scale = 1.0 / cs.df_scale;  // a power of two: exact
  const float s32 = (float)cs.df_scale, inv_s32 = (float)inv_scale;

  PhaseClock clk(cs, tm);
  const bool src_mode = cs.n_corr > 0 || cs.vSu != nullptr || cs.vSp != nullptr;
  const bool fuse = !src_mode;  // verification fused with the next step's T0 (pass V)
  // this step's rows and seed come from the last V pass: of this launch, or of the last
  // launch when it ended with them in place and nothing changed since (flags[1], cleared by
  // the host with every change to the case; read by every CTA before the first barrier)
  bool seeded = fuse && ld_volatile_i32(cs.flags + 1) != 0 && ld_volatile_i32(cs.flags) != 0;
  double seed[3] = {0.0, 0.0, 0.0};  // their team totals: normFactor sum, sum|r|, rho
  if (seeded) {
    seed[0] = __ldcg(cs.seed_sums);
    seed[1] = __ldcg(cs.seed_sums + 1);
    seed[2] = __ldcg(cs.seed_sums + 2);
  }
  bool convert = ld_volatile_i32(cs.flags) == 0;  // read by every CTA before the first barrier
  for (int step = 0; step < n_steps; ++step) {
    int iters_tot = 0, sweeps_tot = 0, status = 0;
    double nf0 = 0.0, init0 = 0.0, res = 0.0;
    bool conv = false;
    for (int pass = 0; pass <= cs.n_corr; ++pass) {
      double xRef = 0.0;
      // x_old holds the step's starting field once S ran (pass 0 saves it, later passes keep
      // it); a seeded step saves it at its first correction
      bool old_saved = !seeded;
      bool have_u = seeded;
      double u[3] = {seed[0], seed[1], seed[2]};
      seeded = false;
      // consumed: constants from here on, so that no register holds them through the sweeps
      seed[0] = seed[1] = seed[2] = 0.0;
      if (have_u == false) {
        // ---- S: sum of x; the step's starting field (T1's ddt term) ------------------
        double v[1] = {pass_sum_df<B>(cref, c0, c1, convert, false, pass == 0)};
        if (!team_allreduce<1>(tm, v, sh)) return false;
        mark_split(cs, tm, convert);
        clk.lap(kPhAssembly);
        xRef = v[0] / (double)cs.N;
      }
      double nf = 0.0, init_res = 0.0;
      int iters = 0, sweeps = 0;
      for (;;) {
        // ---- T0 (rows + true residual) or T1 (true residual after a correction) ----------
        if (!have_u) {
          if (sweeps == 0) {
            const Sums3 ui = src_mode ? pass_rows_init_mixed_df<B, W, true>(cref, c0, c1, xRef, s32, inv_s32)
                                      : pass_rows_init_mixed_df<B, W, false>(cref, c0, c1, xRef, s32, inv_s32);
            u[0] = ui.a;
            u[1] = ui.b;
            u[2] = ui.c;
          } else {
            const double2 ut = src_mode ? pass_true_residual_df<B, W, true>(cref, c0, c1, inv_s32)
                                        : pass_true_residual_df<B, W, false>(cref, c0, c1, inv_s32);
            u[0] = 0.0;
            u[1] = ut.x;
            u[2] = ut.y;
          }
          if (!team_allreduce<3>(tm, u, sh)) return false;
          clk.lap(kPhInit);
        }
        have_u = false;
        if (sweeps == 0) {
          nf = (u[0] + kSmall * cs.df_scale) * inv_scale;
          init_res = u[1] * inv_scale / nf;
        }
        res = u[1] * inv_scale / nf;
        if (!isfinite(res)) {
          status = LFM_ENONFINITE;
          break;
        }
        const bool c_ok = converged(res, init_res, cs.tol, cs.rel_tol);
        if ((c_ok && !(sweeps == 0 && cs.min_iter > 0)) || sweeps == kMaxSweeps || iters >= cs.max_iter) break;

        // ---- inner FP32 CG on A dx = r (unscaled) -----------------------------------------
        const double inner_tol = fmax(cs.tol, kInnerRel * res);
        const int min_inner = sweeps == 0 ? cs.min_iter : 0;
        double rho = u[2], beta = 0.0;
        int k = 0;
        for (;;) {
          if (k > 0) {
            pass_direction<B, float>(c0, c1, (float)beta, p, w);
            if (!team_barrier(tm, sh)) return false;
            clk.lap(kPhP);
          }
          bool m_ok;
          double s1[1] = {amul_dot_f32<B, W>(slots32(cs), c0, c1, p, q, tm, m_ok)};
          if (!m_ok) return false;
          if (!team_allreduce<1>(tm, s1, sh)) return false;
          clk.lap(kPhM);
          const double sigma = s1[0];
          if (fabs(sigma) / nf < kVSmall) {
            status = LFM_ESINGULAR;
            break;
          }
          const double2 su = k == 0 ? pass_update_f32<B, true>(c0, c1, (float)(rho / sigma), dx, r, w, p, q, rD)
                                    : pass_update_f32<B, false>(c0, c1, (float)(rho / sigma), dx, r, w, p, q, rD);
          double s2[2] = {su.x, su.y};
          if (!team_allreduce<2>(tm, s2, sh)) return false;
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
        // ---- C: x += dx --------------------------------------------------------------------
        double sx[1] = {pass_correct_df<B>(cref, c0, c1, !old_saved)};
        if (!team_allreduce<1>(tm, sx, sh)) return false;
        old_saved = true;
        clk.lap(kPhCorrect);
        ++sweeps;
        if (fuse) {
          // ---- V: the verification residual and the next step's T0 -----------------------
          const Sums4 uv = pass_verify_next_df<B, W>(cref, c0, c1, sx[0] / (double)cs.N, s32, inv_s32);
          double v4[4] = {uv.a, uv.b, uv.c, uv.d};
          if (!team_allreduce<4>(tm, v4, sh)) return false;
          clk.lap(kPhInit);
          res = v4[0] * inv_scale / nf;
          if (!isfinite(res)) {
            status = LFM_ENONFINITE;
            break;
          }
          if (converged(res, init_res, cs.tol, cs.rel_tol) || sweeps == kMaxSweeps || iters >= cs.max_iter) {
            seeded = true;  // the step ends with this x: the next one starts from V's rows
            seed[0] = v4[1];
            seed[1] = v4[2];
            seed[2] = v4[3];
            break;
          }
          // another sweep: T1 re-seeds the inner solve from the verification residual
        }
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
      return true;
    }
  }
  // the launch ends: whether the next step's rows and seed are in place, for the next launch
  // (every CTA read flags[1] before the first barrier of this launch)
  if (tm.rank == 0 && tid == 0) {
    if (seeded) {
      cs.seed_sums[0] = seed[0];
      cs.seed_sums[1] = seed[1];
      cs.seed_sums[2] = seed[2];
    }
    *reinterpret_cast<volatile int32_t*>(cs.flags + 1) = seeded ? 1 : 0;
  }
  return true;
}

// The mixed form with df64 outer passes (the case must satisfy mixed_uses_df).
template <int B, int W>
__device__ void run_steps_mixed_df(const CaseDev& cs, const CaseDev& cref, const Team& tm, int n_steps,
                                   TeamShared& sh, int stats_base = 0) {
  if (n_steps <= 0) return;
  int c0, c1;
  cta_range(cs.N, tm.size, tm.rank, c0, c1);
  steps_mixed_df<B, W>(cs, cref, tm, n_steps, sh, stats_base, c0, c1);
  pass_store_x<B>(cref, c0, c1, false);
}

// The mixed form: df64 outer passes where mixed_uses_df, else FP64 ones (lfm_solve.cuh).
template <int B, int W>
__device__ void run_steps_mixed_any(const CaseDev& cs, const CaseDev& cref, const Team& tm, int n_steps, int mode,
                                    TeamShared& sh, int stats_base = 0) {
  if (mode != kModeSteps || !mixed_uses_df(cs))
    run_steps_mixed<B, W>(cs, cref, tm, n_steps, mode, sh, stats_base);
  else
    run_steps_mixed_df<B, W>(cs, cref, tm, n_steps, sh, stats_base);
}

}  // namespace
}  // namespace lfm

// One case decomposed into parts, each with its own vectors: the data flow of the paper's
// multi-GPU runs (section "Evaluation": the mesh decomposed over GPUs, one halo exchange of p
// per PCG iteration and global sums), emulated in one cooperative launch on one GPU.
//
// Decomposition: contiguous ranges of cell labels, as equal as the count allows (on a
// naturally numbered box these are slabs along the last axis, the paper's simple
// decomposition). A part owns the rows of its labels; a neighbour label outside its range is
// a ghost of the part -- one ghost slot per distinct outside label, ordered by label (so by
// source part). Each part's vectors T and p carry their ghosts after the owned entries.
//
// Exchange: the part that owns an interface cell pushes its value into every ghost slot that
// mirrors it, right after computing it -- T once per step (in the pass that sums T for
// xRef), p in every pass that writes p -- and the team barrier that ends the pass makes the
// pushes visible before any part reads its ghosts. A push is a store into another part's
// memory: what one GPU does to a peer's memory over NVLink, or what a send/receive pair
// carries. Global sums (xRef, normFactor, rho, sigma, sum|r|) are the team reductions over
// all parts' CTAs, ordered by part.
//
// A part's rows are the global rows of its labels (the same coefficients, the same
// summation order), so the decomposed step is the single-case FP64 step with the vectors
// split: only the order of the global sums differs.
#include <algorithm>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "lfm_device.cuh"
#include "lfm_internal.h"
#include "lfm_solve.cuh"

namespace lfm {

// ---- plan (host) -----------------------------------------------------------------------

int32_t dd_first_label(int32_t N, int32_t P, int32_t s) { return (int32_t)(((int64_t)N * s) / P); }

int32_t dd_part_of(int32_t N, int32_t P, int32_t label) {
  // largest s with first_label(s) <= label
  int32_t s = (int32_t)(((int64_t)label * P) / N);
  while (s + 1 < P && dd_first_label(N, P, s + 1) <= label) ++s;
  while (s > 0 && dd_first_label(N, P, s) > label) --s;
  return s;
}

// Ghost labels of part s from the neighbour lists of its cells (nbr(c, k) for k < deg(c)),
// sorted ascending and unique.
template <typename Nbr>
static std::vector<int32_t> dd_ghosts(int32_t N, int32_t P, int32_t s, Nbr nbr) {
  const int32_t a = dd_first_label(N, P, s), b = dd_first_label(N, P, s + 1);
  std::vector<int32_t> g;
  for (int32_t c = a; c < b; ++c) nbr(c, [&](int32_t o) {
      if (o < a || o >= b) g.push_back(o);
    });
  std::sort(g.begin(), g.end());
  g.erase(std::unique(g.begin(), g.end()), g.end());
  return g;
}

template <typename Nbr>
static void dd_plan_part(int32_t N, int32_t P, int32_t s, Nbr nbr, DdPlanPart& out) {
  out.first = dd_first_label(N, P, s);
  out.n_owned = dd_first_label(N, P, s + 1) - out.first;
  out.ghost = dd_ghosts(N, P, s, nbr);
  out.send_src.clear();
  out.send_part.clear();
  out.send_slot.clear();
  // what s sends: for every other part t, the ghosts of t that s owns, at t's slots
  struct E {
    int32_t src, part, slot;
  };
  std::vector<E> e;
  for (int32_t t = 0; t < P; ++t) {
    if (t == s) continue;
    const int32_t ta = dd_first_label(N, P, t), tb = dd_first_label(N, P, t + 1);
    // quick reject: t's ghosts lie next to its range; compute them only if s can hold one
    bool adjacent = false;
    for (int32_t c = ta; c < tb && !adjacent; ++c) nbr(c, [&](int32_t o) {
        if (o >= out.first && o < out.first + out.n_owned) adjacent = true;
      });
    if (!adjacent) continue;
    const std::vector<int32_t> tg = dd_ghosts(N, P, t, nbr);
    for (size_t j = 0; j < tg.size(); ++j)
      if (tg[j] >= out.first && tg[j] < out.first + out.n_owned) e.push_back({tg[j] - out.first, t, (int32_t)j});
  }
  std::sort(e.begin(), e.end(), [](const E& x, const E& y) {
    return x.src != y.src ? x.src < y.src : (x.part != y.part ? x.part < y.part : x.slot < y.slot);
  });
  for (const E& x : e) {
    out.send_src.push_back(x.src);
    out.send_part.push_back(x.part);
    out.send_slot.push_back(x.slot);
  }
}

void dd_plan_from_faces(int32_t N, int32_t F, const int32_t* owner, const int32_t* neighbour, int32_t P,
                        int32_t s, DdPlanPart& out) {
  // cell -> neighbour lists (CSR)
  std::vector<int32_t> start(N + 1, 0), list(2 * (size_t)F);
  for (int32_t f = 0; f < F; ++f) {
    ++start[owner[f] + 1];
    ++start[neighbour[f] + 1];
  }
  for (int32_t c = 0; c < N; ++c) start[c + 1] += start[c];
  std::vector<int32_t> fill(start.begin(), start.end() - 1);
  for (int32_t f = 0; f < F; ++f) {
    list[fill[owner[f]]++] = neighbour[f];
    list[fill[neighbour[f]]++] = owner[f];
  }
  dd_plan_part(N, P, s,
               [&](int32_t c, auto&& fn) {
                 for (int32_t i = start[c]; i < start[c + 1]; ++i) fn(list[i]);
               },
               out);
}

void dd_plan_from_slots(int32_t N, int32_t W, const int32_t* slot_other, int32_t P, int32_t s, DdPlanPart& out) {
  dd_plan_part(N, P, s,
               [&](int32_t c, auto&& fn) {
                 for (int32_t k = 0; k < W; ++k) {
                   const int32_t o = slot_other[(size_t)k * N + c];
                   if (o != c) fn(o);
                 }
               },
               out);
}

// ---- the decomposed FP64 step (device) --------------------------------------------------
namespace {

// Pushes v[src] of this CTA's interface cells into the ghost slots that mirror them (the
// CTA's send entries [e0, e1): those whose source cell lies in its own cell range, written by
// its own threads, hence the CTA synchronisation first).
__device__ __forceinline__ void dd_push(const DdPart* __restrict__ parts, const DdPart& me, int e0, int e1, bool x,
                                        int B) {
  __syncthreads();
  const double* __restrict__ v = x ? me.x : me.p;
  for (int e = e0 + (int)threadIdx.x; e < e1; e += B) {
    const DdPart& d = parts[me.send_part[e]];
    double* dst = x ? d.x : d.p;
    dst[d.N + me.send_slot[e]] = v[me.send_src[e]];
  }
}

// The row of owned cell i (global label g = first + i): the global row's coefficients in slot
// order with the part's local column ids, then the boundary faces and V/dt -- the arithmetic
// of assemble_row.
template <int W>
__device__ __forceinline__ Row dd_row(const CaseDev& cs, const DdPart& me, int i) {
  const size_t Ng = (size_t)cs.N, N = (size_t)me.N;
  const int g = me.first + i;
  const double* __restrict__ x = me.x;
  Row o;
  o.xc = x[i];
  double off = 0.0;
  const int ns = W > 0 ? W : cs.W;
  o.d = 0.0;
#pragma unroll
  for (int k = 0; k < (W > 0 ? W : kMaxSlots); ++k) {
    if (W == 0 && k >= ns) break;
    const double u = cs.slot_coef[(size_t)k * Ng + g];
    o.d = k == 0 ? -u : __dadd_rn(o.d, -u);
    off = fma(u, x[me.slot_local[(size_t)k * N + i]], off);
  }
  row_boundary(cs, g, o.xc, o);
  o.ax = fma(o.d, o.xc, off);
  return o;
}

template <int B, int W>
__global__ void __launch_bounds__(B, 1024 / B) dd_step_kernel(CaseDev cs, const DdPart* __restrict__ parts,
                                                              const int32_t* __restrict__ cta_part,
                                                              const int32_t* __restrict__ cta_rank, Launch L,
                                                              int n_steps) {
  __shared__ TeamShared sh;
  __shared__ DdPart me;
  if (threadIdx.x == 0) me = parts[cta_part[blockIdx.x]];
  __syncthreads();
  const Team tm{(int)gridDim.x, (int)blockIdx.x, cs.sync, cs.partials, L.timeout_ns};
  if (threadIdx.x == 0) team_join(tm, sh);
  int c0, c1;
  cta_range(me.N, me.ctas, cta_rank[blockIdx.x], c0, c1);
  // this CTA's send entries: those with source cells in [c0, c1) (send_src ascending)
  int e0 = 0, e1 = 0;
  {
    int lo = 0, hi = me.n_send;
    while (lo < hi) {
      const int m = (lo + hi) >> 1;
      if (me.send_src[m] < c0) lo = m + 1; else hi = m;
    }
    e0 = lo;
    hi = me.n_send;
    while (lo < hi) {
      const int m = (lo + hi) >> 1;
      if (me.send_src[m] < c1) lo = m + 1; else hi = m;
    }
    e1 = lo;
  }
  const int tid = threadIdx.x;
  const size_t Ng = (size_t)cs.N, N = (size_t)me.N;
  for (int step = 0; step < n_steps; ++step) {
    // ---- sum of T (xRef) and the exchange of T's interface values ----------------------
    double v[1] = {0.0};
    for (int c = c0 + tid; c < c1; c += B) v[0] += me.x[c];
    dd_push(parts, me, e0, e1, true, B);
    if (!team_allreduce<1>(tm, v, sh)) return;
    const double xRef = v[0] / (double)cs.N;
    // ---- rows, initial residual, normFactor, first direction (p = w, exchanged) ---------
    double u[3] = {0.0, 0.0, 0.0};
    for (int c = c0 + tid; c < c1; c += B) {
      const Row o = dd_row<W>(cs, me, c);
      const double rd = __drcp_rn(o.d);
      me.diag[c] = o.d;
      me.rD[c] = rd;
      const double rc = o.s - o.ax;
      u[0] += fabs(fma(-o.sa, xRef, o.ax)) + fabs(fma(-o.sa, xRef, o.s));
      u[1] += fabs(rc);
      const double wc = rd * rc;
      u[2] = fma(wc, rc, u[2]);
      me.r[c] = rc;
      me.p[c] = wc;
    }
    dd_push(parts, me, e0, e1, false, B);
    if (!team_allreduce<3>(tm, u, sh)) return;
    const double nf = u[0] + kSmall;
    const double init_res = u[1] / nf;
    double res = init_res, rho = u[2], beta = 0.0;
    int iters = 0, status = 0;
    bool conv = converged(res, init_res, cs.tol, cs.rel_tol);
    if (cs.min_iter > 0 || !conv) {
      for (;;) {
        if (iters > 0) {
          int c = c0 + tid;
          for (; c + B < c1; c += 2 * B) {  // two cells per trip, the next trip prefetched
            pf_next<B>(me.p, c, c1);
            pf_next<B>(me.w, c, c1);
            const double pa = me.p[c], pb = me.p[c + B], wa = me.w[c], wb = me.w[c + B];
            me.p[c] = fma(beta, pa, wa);
            me.p[c + B] = fma(beta, pb, wb);
          }
          if (c < c1) me.p[c] = fma(beta, me.p[c], me.w[c]);
          dd_push(parts, me, e0, e1, false, B);
          if (!team_barrier(tm, sh)) return;
        }
        // q = A p over the owned rows (ghost columns from the exchange), sigma = p.q; with a
        // fixed slot width two rows per trip, all their loads issued first, the matrix with
        // streaming loads (the cells per thread and the order of the sum as one row per trip)
        double s1[1] = {0.0};
        int c = c0 + tid;
        if constexpr (W > 0) {
          for (; c + B < c1; c += 2 * B) {
            const int c2 = c + B;
            const double pc = me.p[c], pc2 = me.p[c2];
            double acc = __ldcs(me.diag + c) * pc, acc2 = __ldcs(me.diag + c2) * pc2;
            int o[W], o2[W];
            double u[W], u2[W];
#pragma unroll
            for (int k = 0; k < W; ++k) {
              o[k] = __ldcs(me.slot_local + (size_t)k * N + c);
              o2[k] = __ldcs(me.slot_local + (size_t)k * N + c2);
              u[k] = __ldcs(cs.slot_coef + (size_t)k * Ng + me.first + c);
              u2[k] = __ldcs(cs.slot_coef + (size_t)k * Ng + me.first + c2);
            }
#pragma unroll
            for (int k = 0; k < W; ++k) {
              acc = fma(u[k], me.p[o[k]], acc);
              acc2 = fma(u2[k], me.p[o2[k]], acc2);
            }
            me.q[c] = acc;
            me.q[c2] = acc2;
            s1[0] = fma(acc, pc, s1[0]);
            s1[0] = fma(acc2, pc2, s1[0]);
          }
        }
        for (; c < c1; c += B) {
          const double pc = me.p[c];
          double acc = me.diag[c] * pc;
          const int ns = W > 0 ? W : cs.W;
#pragma unroll
          for (int k = 0; k < (W > 0 ? W : kMaxSlots); ++k) {
            if (W == 0 && k >= ns) break;
            acc = fma(cs.slot_coef[(size_t)k * Ng + me.first + c], me.p[me.slot_local[(size_t)k * N + c]], acc);
          }
          me.q[c] = acc;
          s1[0] = fma(acc, pc, s1[0]);
        }
        if (!team_allreduce<1>(tm, s1, sh)) return;
        const double sigma = s1[0];
        if (fabs(sigma) / nf < kVSmall) {
          status = LFM_ESINGULAR;
          break;
        }
        const double alpha = rho / sigma;
        double s2[2] = {0.0, 0.0};
        for (int c = c0 + tid; c < c1; c += B) {
          if (c + B < c1) {  // the next trip's cell, into L2
            prefetch_l2(me.q + c + B);
            prefetch_l2(me.r + c + B);
            prefetch_l2(me.p + c + B);
            prefetch_l2(me.x + c + B);
            prefetch_l2(me.rD + c + B);
          }
          const double rn = fma(-alpha, me.q[c], me.r[c]);
          const double wn = me.rD[c] * rn;
          me.x[c] = fma(alpha, me.p[c], me.x[c]);
          me.r[c] = rn;
          me.w[c] = wn;
          s2[0] += fabs(rn);
          s2[1] = fma(wn, rn, s2[1]);
        }
        if (!team_allreduce<2>(tm, s2, sh)) return;
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
    write_stats(cs, tm, step, iters, conv ? 1 : 0, iters > 0 ? 1 : 0, status, init_res, res, nf);
    if (status != 0) {
      if (tm.rank == 0 && tid == 0) set_status(cs.sync, status);
      return;
    }
  }
}

template <int B>
void* dd_fn_w(int W) {
  return W == 6 ? (void*)dd_step_kernel<B, 6> : (void*)dd_step_kernel<B, 0>;
}

}  // namespace

int dd_max_ctas(int threads, int W, int device) {
  void* fn = threads == 256 ? dd_fn_w<256>(W) : threads == 512 ? dd_fn_w<512>(W) : nullptr;
  if (!fn) return 0;
  int per_sm = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, 0) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
  const int n = per_sm * sms;
  return n < kMaxCtas ? n : kMaxCtas;
}

cudaError_t launch_dd_steps(const CaseDev& cs, const DdPart* parts, const int32_t* cta_part, const int32_t* cta_rank,
                            const Launch& L, int n_steps, cudaStream_t stream) {
  void* fn = L.threads == 256 ? dd_fn_w<256>(cs.W) : L.threads == 512 ? dd_fn_w<512>(cs.W) : nullptr;
  if (!fn) return cudaErrorInvalidValue;
  CaseDev a0 = cs;
  const DdPart* a1 = parts;
  const int32_t* a2 = cta_part;
  const int32_t* a3 = cta_rank;
  Launch a4 = L;
  int a5 = n_steps;
  void* args[] = {&a0, &a1, &a2, &a3, &a4, &a5};
  return cudaLaunchCooperativeKernel(fn, dim3(L.ctas), dim3(L.threads), args, 0, stream);
}

}  // namespace lfm

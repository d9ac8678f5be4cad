// Allocation-free PCG solve (lfm_pcg_solve_static in include/lapfoam.h).
//
// Some callers cannot allocate device memory: a plug-in running inside a host code whose
// memory manager owns every device buffer, or a real-time loop that must not call an
// allocator once it has started. This entry point serves them: the caller passes the LDU
// system and the solution vector in device memory it already owns, and every piece of
// working memory the solve needs lives in one file-scope device array declared below.
//
// The array is fixed at load time (every GPU that loads the library holds it until the
// process exits) and shared by all calls: each call re-initialises what must start at zero,
// and two calls whose kernels overlap on a GPU would race on it, so callers must order
// their calls (one stream, or explicit synchronisation).
//
// The solve is the same diagonal-preconditioned CG with the normFactor residual as the
// step kernels, run by one CTA: the face-to-cell lists are rebuilt from owner/neighbour on
// every call (binary search for the owned faces, counting + per-cell sort for the
// neighbour-side faces), then the CG recurrence runs with block-level reductions.
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "lfm_internal.h"

namespace {

constexpr int kThreads = 1024;
constexpr int32_t kMaxCells = lfm::kStaticMaxCells;
constexpr int32_t kMaxFaces = lfm::kStaticMaxFaces;

// Byte layout of the scratch array.
constexpr size_t align256(size_t v) { return (v + 255) / 256 * 256; }
constexpr size_t kOffR = 0;
constexpr size_t kOffW = kOffR + align256(8 * (size_t)kMaxCells);
constexpr size_t kOffP = kOffW + align256(8 * (size_t)kMaxCells);
constexpr size_t kOffQ = kOffP + align256(8 * (size_t)kMaxCells);
constexpr size_t kOffOwnStart = kOffQ + align256(8 * (size_t)kMaxCells);
constexpr size_t kOffLoStart = kOffOwnStart + align256(4 * ((size_t)kMaxCells + 1));
constexpr size_t kOffLoFill = kOffLoStart + align256(4 * ((size_t)kMaxCells + 1));
constexpr size_t kOffLosort = kOffLoFill + align256(4 * (size_t)kMaxCells);
constexpr size_t kOffLoOther = kOffLosort + align256(4 * (size_t)kMaxFaces);
constexpr size_t kOffStats = kOffLoOther + align256(4 * (size_t)kMaxFaces);
constexpr size_t kOffReason = kOffStats + align256(sizeof(lfm_step_stats));
constexpr size_t kScratchBytes = kOffReason + align256(2 * sizeof(int32_t));

// Why the kernel rejected the addressing (first int of the reason words; the second holds a
// face or cell id).
enum Reason { kBadNone = 0, kBadFace = 1, kBadOrder = 2, kBadDegree = 3 };

static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

struct Scratch {
  double *r, *w, *p, *q;
  int32_t *own_start, *lo_start, *lo_fill, *losort, *lo_other;
  lfm_step_stats* stats;
  int32_t* reason;  // [2] Reason and the offending face or cell
};

__device__ __forceinline__ Scratch carve(unsigned char* base) {
  Scratch s;
  s.r = reinterpret_cast<double*>(base + kOffR);
  s.w = reinterpret_cast<double*>(base + kOffW);
  s.p = reinterpret_cast<double*>(base + kOffP);
  s.q = reinterpret_cast<double*>(base + kOffQ);
  s.own_start = reinterpret_cast<int32_t*>(base + kOffOwnStart);
  s.lo_start = reinterpret_cast<int32_t*>(base + kOffLoStart);
  s.lo_fill = reinterpret_cast<int32_t*>(base + kOffLoFill);
  s.losort = reinterpret_cast<int32_t*>(base + kOffLosort);
  s.lo_other = reinterpret_cast<int32_t*>(base + kOffLoOther);
  s.stats = reinterpret_cast<lfm_step_stats*>(base + kOffStats);
  s.reason = reinterpret_cast<int32_t*>(base + kOffReason);
  return s;
}

// Block-wide sum of NS values (fixed shuffle + shared-memory tree: deterministic).
template <int NS>
__device__ __forceinline__ void block_sum(double* v, double* sh /*32*NS + NS*/) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NS; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NS; ++k) sh[warp * NS + k] = v[k];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      double t = sh[lane * NS + k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane == 0) sh[32 * NS + k] = t;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NS; ++k) v[k] = sh[32 * NS + k];
  __syncthreads();
}

__device__ __forceinline__ bool conv_test(double res, double init_res, double tol, double rel_tol) {
  return res < tol || (rel_tol > 0.0 && res < rel_tol * init_res);
}

// Row c of A v from the per-call lists: neighbour-side faces, then owned faces.
__device__ __forceinline__ double row(const Scratch& s, int c, const int32_t* __restrict__ neighbour,
                                      const double* __restrict__ diag, const double* __restrict__ upper,
                                      const double* v) {
  double acc = diag[c] * v[c];
  for (int i = s.lo_start[c]; i < s.lo_start[c + 1]; ++i) acc = fma(upper[s.losort[i]], v[s.lo_other[i]], acc);
  for (int f = s.own_start[c]; f < s.own_start[c + 1]; ++f) acc = fma(upper[f], v[neighbour[f]], acc);
  return acc;
}

__global__ void __launch_bounds__(kThreads) static_pcg_kernel(
    unsigned char* scratch, int32_t N, int32_t F, const int32_t* __restrict__ owner,
    const int32_t* __restrict__ neighbour, const double* __restrict__ diag, const double* __restrict__ upper,
    const double* __restrict__ source, double* __restrict__ x, double tol, double rel_tol, int32_t max_iter,
    int32_t min_iter) {
  __shared__ double sh[32 * 3 + 3];
  __shared__ int32_t s_bad;
  __shared__ int32_t s_warp[32];
  const Scratch s = carve(scratch);
  const int tid = threadIdx.x;
  if (tid == 0) s_bad = 0;
  __syncthreads();

  // ---- face-to-cell lists ---------------------------------------------------------------
  // Nothing read from owner/neighbour is used as an address before it has been checked; a
  // rejected system leaves x untouched.
  for (int f = tid; f < F; f += kThreads) {
    const int32_t o = owner[f], n = neighbour[f];
    const int bad = (o < 0 || n <= o || n >= N) ? kBadFace : (f > 0 && owner[f - 1] > o) ? kBadOrder : kBadNone;
    if (bad && atomicCAS(&s_bad, 0, bad) == 0) s.reason[1] = f;
  }
  for (int c = tid; c < N; c += kThreads) s.lo_fill[c] = 0;
  __syncthreads();
  if (s_bad) {
    if (tid == 0) {
      s.reason[0] = s_bad;
      s.stats->status = LFM_EINVAL;
    }
    return;
  }
  for (int f = tid; f < F; f += kThreads) atomicAdd(&s.lo_fill[neighbour[f]], 1);
  // owned faces: faces are sorted by owner, so own_start[c] = first face with owner >= c
  for (int c = tid; c <= N; c += kThreads) {
    int lo = 0, hi = F;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (owner[mid] < c) lo = mid + 1; else hi = mid;
    }
    s.own_start[c] = lo;
  }
  __syncthreads();
  // at most kMaxSlots internal faces per cell (the limit of the context path): it bounds the
  // per-cell list sort below and every row's work
  for (int c = tid; c < N; c += kThreads)
    if (s.lo_fill[c] + s.own_start[c + 1] - s.own_start[c] > lfm::kMaxSlots && atomicCAS(&s_bad, 0, kBadDegree) == 0)
      s.reason[1] = c;
  __syncthreads();
  if (s_bad) {
    if (tid == 0) {
      s.reason[0] = s_bad;
      s.stats->status = LFM_EINVAL;
    }
    return;
  }
  // exclusive scan of the neighbour-side counts: each thread scans a contiguous run
  const int per = (N + kThreads - 1) / kThreads;
  const int a0 = tid * per, a1 = min(N, a0 + per);
  int run = 0;
  for (int c = a0; c < a1; ++c) run += s.lo_fill[c];
  // block exclusive scan of the run totals
  const int lane = tid & 31, warp = tid >> 5;
  int incl = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int wv = s_warp[lane];
    int wincl = wv;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, wincl, o);
      if (lane >= o) wincl += t;
    }
    s_warp[lane] = wincl - wv;
  }
  __syncthreads();
  int base = s_warp[warp] + incl - run;
  for (int c = a0; c < a1; ++c) {
    s.lo_start[c] = base;
    base += s.lo_fill[c];
    s.lo_fill[c] = 0;
  }
  if (tid == kThreads - 1) s.lo_start[N] = F;
  __syncthreads();
  for (int f = tid; f < F; f += kThreads) {
    const int32_t n = neighbour[f];
    s.losort[s.lo_start[n] + atomicAdd(&s.lo_fill[n], 1)] = f;
  }
  __syncthreads();
  // ascending face order inside each cell's short list (at most kMaxSlots entries), so every
  // run sums in the same order
  for (int c = tid; c < N; c += kThreads) {
    const int b = s.lo_start[c], e = s.lo_start[c + 1];
    for (int i = b + 1; i < e; ++i) {
      const int32_t v = s.losort[i];
      int j = i - 1;
      while (j >= b && s.losort[j] > v) {
        s.losort[j + 1] = s.losort[j];
        --j;
      }
      s.losort[j + 1] = v;
    }
    for (int i = b; i < e; ++i) s.lo_other[i] = owner[s.losort[i]];
  }
  __syncthreads();

  // ---- initial residual and normFactor -------------------------------------------------
  double v1[1] = {0.0};
  for (int c = tid; c < N; c += kThreads) v1[0] += x[c];
  block_sum<1>(v1, sh);
  const double xRef = v1[0] / (double)N;
  double u[3] = {0.0, 0.0, 0.0};
  for (int c = tid; c < N; c += kThreads) {
    const double ax = row(s, c, neighbour, diag, upper, x);
    double rs = diag[c];
    for (int i = s.lo_start[c]; i < s.lo_start[c + 1]; ++i) rs += upper[s.losort[i]];
    for (int f = s.own_start[c]; f < s.own_start[c + 1]; ++f) rs += upper[f];
    const double b = source[c];
    const double rc = b - ax;
    const double pA = rs * xRef;
    u[0] += fabs(ax - pA) + fabs(b - pA);
    u[1] += fabs(rc);
    const double wc = (1.0 / diag[c]) * rc;
    u[2] = fma(wc, rc, u[2]);
    s.r[c] = rc;
    s.p[c] = wc;
  }
  block_sum<3>(u, sh);
  const double nf = u[0] + 1e-20;
  const double init_res = u[1] / nf;
  double res = init_res, rho = u[2], beta = 0.0;
  int iters = 0, status = 0;
  if (min_iter > 0 || !conv_test(res, init_res, tol, rel_tol)) {
    for (;;) {
      if (iters > 0) {
        for (int c = tid; c < N; c += kThreads) s.p[c] = fma(beta, s.p[c], s.w[c]);
        __syncthreads();
      }
      double s1[1] = {0.0};
      for (int c = tid; c < N; c += kThreads) {
        const double qc = row(s, c, neighbour, diag, upper, s.p);
        s.q[c] = qc;
        s1[0] = fma(qc, s.p[c], s1[0]);
      }
      block_sum<1>(s1, sh);
      if (fabs(s1[0]) / nf < 1e-300) {
        status = LFM_ESINGULAR;
        break;
      }
      const double alpha = rho / s1[0];
      double s2[2] = {0.0, 0.0};
      for (int c = tid; c < N; c += kThreads) {
        x[c] = fma(alpha, s.p[c], x[c]);
        const double rc = fma(-alpha, s.q[c], s.r[c]);
        const double wc = (1.0 / diag[c]) * rc;
        s.r[c] = rc;
        s.w[c] = wc;
        s2[0] += fabs(rc);
        s2[1] = fma(wc, rc, s2[1]);
      }
      block_sum<2>(s2, sh);
      res = s2[0] / nf;
      beta = s2[1] / rho;
      rho = s2[1];
      ++iters;
      if (!isfinite(res)) {
        status = LFM_ENONFINITE;
        break;
      }
      const bool cv = conv_test(res, init_res, tol, rel_tol);
      if (!((iters < max_iter && !cv) || iters < min_iter)) break;
    }
  }
  if (tid == 0) {
    lfm_step_stats st;
    st.iters = iters;
    st.converged = conv_test(res, init_res, tol, rel_tol) ? 1 : 0;
    st.sweeps = iters > 0 ? 1 : 0;
    st.status = status;
    st.init_res = init_res;
    st.final_res = res;
    st.norm_factor = nf;
    *s.stats = st;
  }
}

// Device address of the scratch array, looked up once per device (with that device
// current) on the first call made on it.
constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char* g_scratch_ptr[kMaxDevices] = {};

int scratch_for_current_device(unsigned char** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LFM_ECUDA;
  std::lock_guard<std::mutex> lk(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) return LFM_ECUDA;
    g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_ptr[dev];
  return LFM_OK;
}

}  // namespace

namespace {

// Whether the byte ranges [a, a + na) and [b, b + nb) overlap.
bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
  const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  return na > 0 && nb > 0 && x < y + nb && y < x + na;
}

}  // namespace

extern "C" int lfm_pcg_solve_static(int32_t n_cells, int32_t n_faces, const int32_t* owner,
                                    const int32_t* neighbour, const double* diag, const double* upper,
                                    const double* source, double* x, const lfm_solver_opts* opts,
                                    lfm_step_stats* stats, void* cuda_stream) {
  using lfm::set_last_error;
  const char* me = "lfm_pcg_solve_static";
  if (n_cells <= 0 || n_faces < 0)
    return set_last_error(LFM_EINVAL, "%s: n_cells = %d, n_faces = %d (need n_cells > 0, n_faces >= 0)", me, n_cells,
                          n_faces);
  if (n_cells > kMaxCells || n_faces > kMaxFaces)
    return set_last_error(LFM_EINVAL, "%s: %d cells, %d faces exceed the fixed limits of %d cells and %d faces", me,
                          n_cells, n_faces, kMaxCells, kMaxFaces);
  if (!diag || !source || !x || !opts || (n_faces > 0 && (!owner || !neighbour || !upper)))
    return set_last_error(LFM_EINVAL, "%s: a required pointer is NULL", me);
  if (!(opts->tol >= 0) || !(opts->rel_tol >= 0) || opts->max_iter < 1 || opts->min_iter < 0 ||
      opts->min_iter > opts->max_iter || opts->precision != LFM_FP64)
    return set_last_error(LFM_EINVAL,
                          "%s: solver options (tol %g, rel_tol %g, max_iter %d, min_iter %d, precision %d) invalid; "
                          "precision must be LFM_FP64",
                          me, opts->tol, opts->rel_tol, opts->max_iter, opts->min_iter, opts->precision);
  const size_t xb = sizeof(double) * (size_t)n_cells;
  if (overlaps(x, xb, source, xb) || overlaps(x, xb, diag, xb) ||
      overlaps(x, xb, upper, sizeof(double) * (size_t)n_faces) ||
      overlaps(x, xb, owner, sizeof(int32_t) * (size_t)n_faces) ||
      overlaps(x, xb, neighbour, sizeof(int32_t) * (size_t)n_faces))
    return set_last_error(LFM_EINVAL, "%s: x overlaps an input array (the solve is not in place)", me);
  {
    // the call reads its record back and synchronises: it can never be part of a capture
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    const cudaError_t ce = cudaStreamIsCapturing(static_cast<cudaStream_t>(cuda_stream), &cap);
    if (ce != cudaSuccess) {
      cudaGetLastError();
      return set_last_error(LFM_ECUDA, "%s: querying the stream: %s", me, cudaGetErrorString(ce));
    }
    if (cap != cudaStreamCaptureStatusNone)
      return set_last_error(LFM_ESTATE, "%s: the stream is being captured; this call synchronises and cannot be captured",
                            me);
  }
  unsigned char* scratch = nullptr;
  if (scratch_for_current_device(&scratch) != LFM_OK)
    return set_last_error(LFM_ECUDA, "%s: device address of the fixed working array not available", me);
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  lfm_step_stats* dev_stats = reinterpret_cast<lfm_step_stats*>(scratch + kOffStats);
  cudaError_t e;
  // the status and reason words must start at zero for every call
  if ((e = cudaMemsetAsync(scratch + kOffStats, 0, kScratchBytes - kOffStats, stream)) != cudaSuccess)
    return set_last_error(LFM_ECUDA, "%s: clearing the status words: %s", me, cudaGetErrorString(e));
  static_pcg_kernel<<<1, kThreads, 0, stream>>>(scratch, n_cells, n_faces, owner, neighbour, diag, upper, source,
                                                x, opts->tol, opts->rel_tol, opts->max_iter, opts->min_iter);
  if ((e = cudaGetLastError()) != cudaSuccess)
    return set_last_error(LFM_ECUDA, "%s: kernel launch: %s", me, cudaGetErrorString(e));
  lfm_step_stats st;
  int32_t reason[2] = {0, 0};
  if ((e = cudaMemcpyAsync(&st, dev_stats, sizeof st, cudaMemcpyDeviceToHost, stream)) != cudaSuccess ||
      (e = cudaMemcpyAsync(reason, scratch + kOffReason, sizeof reason, cudaMemcpyDeviceToHost, stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(stream)) != cudaSuccess)
    return set_last_error(LFM_ECUDA, "%s: %s", me, cudaGetErrorString(e));
  if (stats) *stats = st;
  switch (st.status) {
    case LFM_OK: return LFM_OK;
    case LFM_EINVAL:
      if (reason[0] == kBadFace)
        return set_last_error(LFM_EINVAL, "%s: face %d: owner/neighbour out of range or owner >= neighbour", me,
                              reason[1]);
      if (reason[0] == kBadOrder)
        return set_last_error(LFM_EINVAL, "%s: faces not sorted by owner at face %d", me, reason[1]);
      return set_last_error(LFM_EINVAL, "%s: cell %d has more than %d internal faces", me, reason[1], lfm::kMaxSlots);
    case LFM_ESINGULAR: return set_last_error(LFM_ESINGULAR, "%s: singular system (p.Ap / normFactor < 1e-300)", me);
    case LFM_ENONFINITE: return set_last_error(LFM_ENONFINITE, "%s: non-finite residual", me);
    default: return set_last_error(st.status, "%s: solver status %d", me, st.status);
  }
}

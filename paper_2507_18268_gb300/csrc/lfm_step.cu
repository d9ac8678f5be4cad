// Single-case persistent cooperative kernels: one launch runs n implicit-Euler steps of
// one case with every CTA of the grid in its team (the step itself is in lfm_solve.cuh).
#include <cuda_runtime.h>

#include <mutex>
#include <utility>
#include <vector>

#include "lfm_device.cuh"
#include "lfm_internal.h"
#include "lfm_solve.cuh"
#include "lfm_solve_df.cuh"
#include "lfm_solve_mixed_df.cuh"

namespace lfm {
namespace {

// ---- kernels ---------------------------------------------------------------------------
template <int B, int W>
__global__ void __launch_bounds__(B, 1024 / B) step_kernel_f64(CaseDev cs, Launch L, int n_steps, int mode) {
  __shared__ TeamShared sh;
  __shared__ CaseDev s_cs;  // addressable copy for the per-step passes
  if ((int)blockIdx.x == L.skip_cta) return;  // test hook: never arrive
  if (threadIdx.x == 0) s_cs = cs;
  __syncthreads();
  const Team tm{(int)gridDim.x, (int)blockIdx.x, cs.sync, cs.partials, L.timeout_ns};
  if (threadIdx.x == 0) team_join(tm, sh);
  run_steps_f64<B, W>(cs, s_cs, tm, n_steps, mode, sh);
}

template <int B, int W>
__global__ void __launch_bounds__(B, 1024 / B) step_kernel_mixed(CaseDev cs, Launch L, int n_steps, int mode) {
  __shared__ TeamShared sh;
  __shared__ CaseDev s_cs;  // addressable copy for the per-step passes
  if ((int)blockIdx.x == L.skip_cta) return;
  if (threadIdx.x == 0) s_cs = cs;
  __syncthreads();
  const Team tm{(int)gridDim.x, (int)blockIdx.x, cs.sync, cs.partials, L.timeout_ns};
  if (threadIdx.x == 0) team_join(tm, sh);
  run_steps_mixed<B, W>(cs, s_cs, tm, n_steps, mode, sh);
}

// The mixed form with df64 outer passes (orthogonal meshes; the host chooses it).
template <int B, int W>
__global__ void __launch_bounds__(B, 1024 / B) step_kernel_mixed_df(CaseDev cs, Launch L, int n_steps, int mode) {
  __shared__ TeamShared sh;
  __shared__ CaseDev s_cs;
  if ((int)blockIdx.x == L.skip_cta) return;
  if (threadIdx.x == 0) s_cs = cs;
  __syncthreads();
  const Team tm{(int)gridDim.x, (int)blockIdx.x, cs.sync, cs.partials, L.timeout_ns};
  if (threadIdx.x == 0) team_join(tm, sh);
  run_steps_mixed_df<B, W>(cs, s_cs, tm, n_steps, sh);
}

template <int B, int W, bool kGeom>
__global__ void __launch_bounds__(B, 1024 / B) step_kernel_df64(CaseDev cs, Launch L, int n_steps, int mode) {
  __shared__ TeamShared sh;
  __shared__ CaseDev s_cs;  // addressable copy for the per-step passes
  if ((int)blockIdx.x == L.skip_cta) return;
  if (threadIdx.x == 0) s_cs = cs;
  __syncthreads();
  const Team tm{(int)gridDim.x, (int)blockIdx.x, cs.sync, cs.partials, L.timeout_ns};
  if (threadIdx.x == 0) team_join(tm, sh);
  run_steps_df64<B, W, kGeom>(cs, s_cs, tm, n_steps, sh);
}

// Set-up (a0): per face g = (DT |Sf|) deltaCoeff (the assembly's products, in its order),
// stored as -g at the face's slot in its owner's and its neighbour's row of the FP64 (and,
// present, FP32) slot arrays. Padding slots keep the zero written at upload.
__global__ void coef_kernel(CaseDev cs) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f < cs.F) {
    const uint2 a0 = reinterpret_cast<const uint2*>(cs.face_slots)[f];
    const uint2 at = make_uint2(LFM_IDX(a0.x, cs.W * cs.N, 0, kChkFaceSlot), LFM_IDX(a0.y, cs.W * cs.N, 0, kChkFaceSlot));
    const double DTf = cs.DT_is_uniform ? cs.DT_uniform : cs.DT[f];
    const double g = __dmul_rn(__dmul_rn(DTf, cs.magSf[f]), cs.delta[f]);
    cs.slot_coef[at.x] = -g;
    cs.slot_coef[at.y] = -g;
    if (cs.slot_coef32) {
      cs.slot_coef32[at.x] = (float)(-g);
      cs.slot_coef32[at.y] = (float)(-g);
    }
  }
}

// df64 set-up (a0): per face g = (DT |Sf|) deltaCoeff in FP64 (the FP64 assembly's order)
// times the case scale, split into a double-float pair and stored at the face's slot in
// its owner's and its neighbour's row (padding slots are cleared before).
__global__ void df_coef_kernel(CaseDev cs, float2* __restrict__ g2) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= cs.F) return;
  const uint2 a0 = reinterpret_cast<const uint2*>(cs.face_slots)[f];
  const uint2 at = make_uint2(LFM_IDX(a0.x, cs.W * cs.N, 0, kChkFaceSlot), LFM_IDX(a0.y, cs.W * cs.N, 0, kChkFaceSlot));
  const double DTf = cs.DT_is_uniform ? cs.DT_uniform : cs.DT[f];
  const double g = __dmul_rn(__dmul_rn(__dmul_rn(DTf, cs.magSf[f]), cs.delta[f]), cs.df_scale);
  const df v = df_from_double(g);
  st_df(g2 + at.x, v);
  st_df(g2 + at.y, v);
}

// df64 operator weights of the general-geometry path: gE and (times the case scale) cK, cL as
// pairs; the closure weight gZ = gD + sum_k gE_k + sum_fixedValue bSf / V in FP64, so that
// G_c = sum_k gE_k (T_k - T_c) + sum_fixedValue (bSf / V)(T_b - T_c) + gZ T_c equals the
// operator form gD T_c + gH + sum_k gE_k T_k.
__global__ void df_ops_kernel(CaseDev cs, float2* __restrict__ E2, float2* __restrict__ K2, float2* __restrict__ L2,
                              float2* __restrict__ Z) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cs.N) return;
  const size_t N = (size_t)cs.N, WN = (size_t)cs.W * N;
  const double s = cs.df_scale;
  double z[3] = {cs.gD[c], cs.gD[N + c], cs.gD[2 * N + c]};
  for (int q = 0; q < 3; ++q) {
    const df v = df_from_double(cs.cK[q * N + c] * s);
    K2[q * N + c] = make_float2(v.hi, v.lo);
  }
  for (int k = 0; k < cs.W; ++k) {
    const size_t at = (size_t)k * N + c;
    for (int q = 0; q < 3; ++q) {
      const double e = cs.gE[q * WN + at];
      z[q] += e;
      const df ev = df_from_double(e), lv = df_from_double(cs.cL[q * WN + at] * s);
      E2[q * WN + at] = make_float2(ev.hi, ev.lo);
      L2[q * WN + at] = make_float2(lv.hi, lv.lo);
    }
  }
  const double rv = 1.0 / cs.V[c];
  for (int k = cs.b_start[c]; k < cs.b_start[c + 1]; ++k) {
    const int bf = LFM_IDX(cs.b_face[k], cs.NB, 0, kChkBFace);
    if (cs.btype[bf] == LFM_FIXED_VALUE)
      for (int q = 0; q < 3; ++q) z[q] += cs.bSf[3 * (size_t)bf + q] * rv;
  }
  for (int q = 0; q < 3; ++q) {
    const df v = df_from_double(z[q]);
    Z[q * N + c] = make_float2(v.hi, v.lo);
  }
}

__global__ void df_vdt_kernel(CaseDev cs, float2* __restrict__ vdt2) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < cs.N) st_df(vdt2 + c, df_from_double(__dmul_rn(cs.vdt[c], cs.df_scale)));
}

__global__ void boundary_values_kernel(CaseDev cs, double* Tb) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < cs.NB) Tb[b] = cs.btype[b] == LFM_FIXED_VALUE ? cs.bval[b] : cs.x[LFM_IDX(cs.bcell[b], cs.N, 0, kChkBFace)];
}

// Gauss gradient of the current T per cell (into cs.grad, component-major).
__global__ void grad_cells_kernel(CaseDev cs) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < cs.N) {
    double g[3];
    op_grad<0>(cs, c, cs.x, g);
    cs.grad[c] = g[0];
    cs.grad[(size_t)cs.N + c] = g[1];
    cs.grad[2 * (size_t)cs.N + c] = g[2];
  }
}

// Boundary values of the gradient (correctBoundaryConditions): the cell's gradient with its
// normal component replaced by the patch snGrad ((T_b - T_P) deltaCoeff for fixedValue, 0
// for zeroGradient).
__global__ void grad_boundary_kernel(CaseDev cs, double* __restrict__ bgrad) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < cs.NB) {
    const size_t N = (size_t)cs.N;
    const int c = LFM_IDX(cs.bcell[b], cs.N, 0, kChkBFace);
    const double* s = cs.bSf + 3 * (size_t)b;
    const double mag = sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
    const double n0 = s[0] / mag, n1 = s[1] / mag, n2 = s[2] / mag;
    const double g0 = cs.grad[c], g1 = cs.grad[N + c], g2 = cs.grad[2 * N + c];
    const double sn = cs.btype[b] == LFM_FIXED_VALUE ? (cs.bval[b] - cs.x[c]) * cs.bdelta[b] : 0.0;
    const double gn = n0 * g0 + n1 * g1 + n2 * g2;
    bgrad[3 * (size_t)b] = g0 + n0 * (sn - gn);
    bgrad[3 * (size_t)b + 1] = g1 + n1 * (sn - gn);
    bgrad[3 * (size_t)b + 2] = g2 + n2 * (sn - gn);
  }
}

// Gradient weights of the slots' other cells (geometry only): the Gauss sum
// V G_c = sum_faces +-Sf (w T_P + (1 - w) T_N) + sum_boundary bSf T_b gives the other cell of
// an owned face the weight (1 - w) Sf and of a neighbour-side face -w Sf; divided by V.
__global__ void grad_weights_kernel(CaseDev cs, double* __restrict__ E) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cs.N) return;
  const size_t N = (size_t)cs.N, WN = (size_t)cs.W * N;
  const double rv = 1.0 / cs.V[c];
  for (int k = 0; k < cs.W; ++k) {
    const size_t at = (size_t)k * N + c;
    const int f = cs.slot_face[at] < 0 ? -1 : LFM_IDX(cs.slot_face[at], cs.F, 0, kChkFaceSlot);
    double e0 = 0.0, e1 = 0.0, e2 = 0.0;
    if (f >= 0) {
      const double w = cs.fw[f];
      const double coef = (cs.slot_other[at] > c ? 1.0 - w : -w) * rv;
      e0 = coef * cs.Sf[3 * (size_t)f];
      e1 = coef * cs.Sf[3 * (size_t)f + 1];
      e2 = coef * cs.Sf[3 * (size_t)f + 2];
    }
    E[at] = e0;
    E[WN + at] = e1;
    E[2 * WN + at] = e2;
  }
}

// The case's operator weights: the gradient's own-cell weight gD (w Sf for owned faces,
// -(1 - w) Sf for neighbour-side faces, bSf for zeroGradient boundary faces) and constant gH
// (bSf T_b for fixedValue faces), both divided by V; and the correction weights: with the
// face flux a.G_P + b.G_N, a = w DT|Sf| k, b = (1 - w) DT|Sf| k, the row gets +a.G_c + b.G_other
// for an owned face and -(b.G_c + a.G_other) for a neighbour-side face.
__global__ void case_ops_kernel(CaseDev cs, double* __restrict__ D, double* __restrict__ H, double* __restrict__ K,
                                double* __restrict__ L) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cs.N) return;
  const size_t N = (size_t)cs.N, WN = (size_t)cs.W * N;
  double d[3] = {0.0, 0.0, 0.0}, h[3] = {0.0, 0.0, 0.0}, kk[3] = {0.0, 0.0, 0.0};
  for (int k = 0; k < cs.W; ++k) {
    const size_t at = (size_t)k * N + c;
    const int f = cs.slot_face[at] < 0 ? -1 : LFM_IDX(cs.slot_face[at], cs.F, 0, kChkFaceSlot);
    double l[3] = {0.0, 0.0, 0.0};
    if (f >= 0) {
      const double w = cs.fw[f];
      const double gam = (cs.DT_is_uniform ? cs.DT_uniform : cs.DT[f]) * cs.magSf[f];
      const bool own = cs.slot_other[at] > c;
      for (int q = 0; q < 3; ++q) {
        const double sf = cs.Sf[3 * (size_t)f + q];
        const double kv = cs.corr[3 * (size_t)f + q];
        const double a = (w * gam) * kv, bb = ((1.0 - w) * gam) * kv;
        if (own) {
          d[q] += w * sf;
          kk[q] += a;
          l[q] = bb;
        } else {
          d[q] -= (1.0 - w) * sf;
          kk[q] -= bb;
          l[q] = -a;
        }
      }
    }
    L[at] = l[0];
    L[WN + at] = l[1];
    L[2 * WN + at] = l[2];
  }
  for (int k = cs.b_start[c]; k < cs.b_start[c + 1]; ++k) {
    const int bf = LFM_IDX(cs.b_face[k], cs.NB, 0, kChkBFace);
    const bool fv = cs.btype[bf] == LFM_FIXED_VALUE;
    for (int q = 0; q < 3; ++q) {
      const double s = cs.bSf[3 * (size_t)bf + q];
      if (fv)
        h[q] += s * cs.bval[bf];
      else
        d[q] += s;
    }
  }
  const double rv = 1.0 / cs.V[c];
  for (int q = 0; q < 3; ++q) {
    D[q * N + c] = d[q] * rv;
    H[q * N + c] = h[q] * rv;
    K[q * N + c] = kk[q];
  }
}

// Face diffusivities from a cell field (the dotInterpolate form of the paper's listing):
// internal faces w (DT_P - DT_N) + DT_N, owner and neighbour from the face's two slots;
// boundary faces the value of their cell. Products and sums rounded separately.
__global__ void dt_cells_kernel(CaseDev cs, const double* __restrict__ DTc, const double* __restrict__ w,
                                double* __restrict__ DTf, double* __restrict__ DTb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < cs.F) {
    const uint2 a0 = reinterpret_cast<const uint2*>(cs.face_slots)[i];
    const uint2 at = make_uint2(LFM_IDX(a0.x, cs.W * cs.N, 0, kChkFaceSlot), LFM_IDX(a0.y, cs.W * cs.N, 0, kChkFaceSlot));
    const double dP = DTc[LFM_IDX(cs.slot_other[at.y], cs.N, 0, kChkSlotCell)];
    const double dN = DTc[LFM_IDX(cs.slot_other[at.x], cs.N, 0, kChkSlotCell)];
    DTf[i] = __dadd_rn(__dmul_rn(w[i], __dsub_rn(dP, dN)), dN);
  }
  if (i < cs.NB) DTb[i] = DTc[LFM_IDX(cs.bcell[i], cs.N, 0, kChkBFace)];
}

__global__ void times_volume_kernel(const double* __restrict__ V, const double* __restrict__ a,
                                    double* __restrict__ out, int n) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < n) out[c] = a ? __dmul_rn(V[c], a[c]) : 0.0;
}

__global__ void vdt_kernel(const double* __restrict__ V, double dt, double* __restrict__ vdt, int n) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < n) vdt[c] = V[c] / dt;
}

__global__ void fill_kernel(double* a, size_t n, double v) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (; i < n; i += stride) a[i] = v;
}

// Kernel-choice codes beside the public precisions: the mixed form with df64 outer passes,
// and the df64 form on general geometry (the orthogonal df64 kernel carries no gradient phase).
constexpr int kMixedDf = 100;
constexpr int kDf64Geom = 101;

template <int B>
void* step_fn_w(int precision, int W) {
  if (W == 6) {
    if (precision == kMixedDf) return (void*)step_kernel_mixed_df<B, 6>;
    if (precision == LFM_MIXED) return (void*)step_kernel_mixed<B, 6>;
    if (precision == kDf64Geom) return (void*)step_kernel_df64<B, 6, true>;
    if (precision == LFM_DF64) return (void*)step_kernel_df64<B, 6, false>;
    return (void*)step_kernel_f64<B, 6>;
  }
  if (precision == kMixedDf) return (void*)step_kernel_mixed_df<B, 0>;
  if (precision == LFM_MIXED) return (void*)step_kernel_mixed<B, 0>;
  if (precision == kDf64Geom) return (void*)step_kernel_df64<B, 0, true>;
  if (precision == LFM_DF64) return (void*)step_kernel_df64<B, 0, false>;
  return (void*)step_kernel_f64<B, 0>;
}

void* step_fn_for(int precision, int threads, int W) {
  switch (threads) {
    case 256: return step_fn_w<256>(precision, W);
    case 512: return step_fn_w<512>(precision, W);
    case 1024: return step_fn_w<1024>(precision, W);
    default: return nullptr;
  }
}

// Dynamic shared memory of a step kernel: the two stages of the bulk-staged FP32 A p of the
// mixed form on orthogonal meshes (the kernel with df64 outer passes, specialised for six
// slots). The mixed kernel for general meshes runs without them: the shared memory comes out
// of the same on-chip array as L1, and its gradient and corrected-row passes, which gather
// through L1, lost more (skewed200: 0.71 -> 0.86 and 1.97 -> 2.01 ms per step) than its A p
// gained (0.655 -> 0.638).
unsigned step_dyn_smem(int precision, int threads, int W) {
  if (precision == kMixedDf && W == 6) {
    switch (threads) {
      case 256: return stage_bytes_f32<256, 6>();
      case 512: return stage_bytes_f32<512, 6>();
      case 1024: return stage_bytes_f32<1024, 6>();
      default: return 0;
    }
  }
  return 0;
}

int per_sm_ctas(int precision, int threads, int W) {
  void* fn = step_fn_for(precision, threads, W);
  if (!fn) return 0;
  const unsigned dyn = step_dyn_smem(precision, threads, W);
  int per_sm = 0;
  if (allow_dyn_smem(fn, dyn) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, dyn) != cudaSuccess)
    return 0;
  return per_sm;
}

}  // namespace

// Opts a kernel into more than 48 KB of dynamic shared memory, once per kernel and device.
cudaError_t allow_dyn_smem(void* fn, unsigned bytes) {
  if (bytes <= 48u * 1024u) return cudaSuccess;
  static std::mutex mu;
  static std::vector<std::pair<void*, int>> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  for (const auto& d : done)
    if (d.first == fn && d.second == dev) return cudaSuccess;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) done.emplace_back(fn, dev);
  return e;
}

int max_coresident_ctas(int precision, int threads, int W, int device) {
  int sms = 0;
  int per_sm = per_sm_ctas(precision, threads, W);
  if (per_sm > 0 && (precision == LFM_MIXED || precision == LFM_DF64)) {  // either kernel of the form may run
    const int per_sm_2 = per_sm_ctas(precision == LFM_MIXED ? kMixedDf : kDf64Geom, threads, W);
    if (per_sm_2 < per_sm) per_sm = per_sm_2;
  }
  if (per_sm <= 0) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
  int n = per_sm * sms;
  return n < kMaxCtas ? n : kMaxCtas;
}

cudaError_t launch_steps(const CaseDev& cs, const Launch& L, int n_steps, int mode,
                         cudaStream_t stream) {
  // matrix read-back of a df64 case runs the FP64 assembly (its arrays are the ones read)
  int prec = (mode == kModeAssembleOnly && cs.precision == LFM_DF64) ? LFM_FP64 : cs.precision;
  // the mixed form runs its outer passes in df64 when the case allows (see mixed_uses_df)
  const bool mixed_df = prec == LFM_MIXED && mode == kModeSteps && mixed_runs_df(cs);
  const bool df_geom = prec == LFM_DF64 && cs.Sf != nullptr;
  const int kind = mixed_df ? kMixedDf : (df_geom ? kDf64Geom : prec);
  void* fn = step_fn_for(kind, L.threads, cs.W);
  if (!fn) return cudaErrorInvalidValue;
  const unsigned dyn = L.stage_rows ? step_dyn_smem(kind, L.threads, cs.W) : 0u;
  const cudaError_t e = allow_dyn_smem(fn, dyn);
  if (e != cudaSuccess) return e;
  CaseDev a0 = cs;
  a0.precision = prec;
  Launch a1 = L;
  int a2 = n_steps, a3 = mode;
  void* args[] = {&a0, &a1, &a2, &a3};
  if (L.skip_copy_cta >= 0) {  // test hook, for this launch only
    const int none = -1;
    cudaError_t he = cudaMemcpyToSymbolAsync(g_skip_copy_cta, &L.skip_copy_cta, sizeof(int), 0,
                                             cudaMemcpyHostToDevice, stream);
    if (he != cudaSuccess) return he;
    he = cudaLaunchCooperativeKernel(fn, dim3(L.ctas), dim3(L.threads), args, dyn, stream);
    const cudaError_t re =
        cudaMemcpyToSymbolAsync(g_skip_copy_cta, &none, sizeof(int), 0, cudaMemcpyHostToDevice, stream);
    return he != cudaSuccess ? he : re;
  }
  return cudaLaunchCooperativeKernel(fn, dim3(L.ctas), dim3(L.threads), args, dyn, stream);
}

bool mixed_runs_df(const CaseDev& cs) {
  return cs.x2 != nullptr && cs.Sf == nullptr && cs.df_scale >= 0x1p-100 && cs.df_scale <= 0x1p100;
}

cudaError_t launch_coef_setup(const CaseDev& cs, cudaStream_t stream) {
  if (cs.F > 0) coef_kernel<<<(cs.F + 255) / 256, 256, 0, stream>>>(cs);
  return cudaGetLastError();
}

cudaError_t launch_df_setup(const CaseDev& cs, cudaStream_t stream) {
  if (!cs.g2 || !cs.vdt2) return cudaErrorInvalidValue;
  float2* g2 = const_cast<float2*>(cs.g2);
  const size_t WN = (size_t)cs.W * cs.N;
  if (WN > 0) {
    cudaError_t e = cudaMemsetAsync(g2, 0, sizeof(float2) * WN, stream);
    if (e != cudaSuccess) return e;
  }
  if (cs.F > 0) df_coef_kernel<<<(cs.F + 255) / 256, 256, 0, stream>>>(cs, g2);
  df_vdt_kernel<<<(cs.N + 255) / 256, 256, 0, stream>>>(cs, const_cast<float2*>(cs.vdt2));
  if (cs.Sf && cs.gE2)
    df_ops_kernel<<<(cs.N + 255) / 256, 256, 0, stream>>>(cs, const_cast<float2*>(cs.gE2), const_cast<float2*>(cs.cK2),
                                                          const_cast<float2*>(cs.cL2), const_cast<float2*>(cs.gZ));
  return cudaGetLastError();
}

cudaError_t launch_geom_ops(const CaseDev& cs, bool with_E, cudaStream_t stream) {
  if (!cs.Sf || cs.N == 0) return cudaErrorInvalidValue;
  const unsigned blocks = (unsigned)((cs.N + 255) / 256);
  if (with_E) grad_weights_kernel<<<blocks, 256, 0, stream>>>(cs, const_cast<double*>(cs.gE));
  case_ops_kernel<<<blocks, 256, 0, stream>>>(cs, const_cast<double*>(cs.gD), const_cast<double*>(cs.gH),
                                              const_cast<double*>(cs.cK), const_cast<double*>(cs.cL));
  return cudaGetLastError();
}

cudaError_t launch_dt_cells(const CaseDev& cs, const double* DTc, const double* w, double* DTf, double* DTb,
                            cudaStream_t stream) {
  const int n = cs.F > cs.NB ? cs.F : cs.NB;
  if (n == 0) return cudaSuccess;
  dt_cells_kernel<<<(n + 255) / 256, 256, 0, stream>>>(cs, DTc, w, DTf, DTb);
  return cudaGetLastError();
}

cudaError_t launch_times_volume(const CaseDev& cs, const double* a, double* out, cudaStream_t stream) {
  times_volume_kernel<<<(cs.N + 255) / 256, 256, 0, stream>>>(cs.V, a, out, cs.N);
  return cudaGetLastError();
}

cudaError_t launch_grad(const CaseDev& cs, double* bgrad, cudaStream_t stream) {
  if (!cs.Sf || !cs.grad) return cudaErrorInvalidValue;
  grad_cells_kernel<<<(cs.N + 255) / 256, 256, 0, stream>>>(cs);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || !bgrad || cs.NB == 0) return e;
  grad_boundary_kernel<<<(cs.NB + 255) / 256, 256, 0, stream>>>(cs, bgrad);
  return cudaGetLastError();
}

cudaError_t launch_boundary_values(const CaseDev& cs, double* Tb, cudaStream_t stream) {
  if (cs.NB == 0) return cudaSuccess;
  boundary_values_kernel<<<(cs.NB + 255) / 256, 256, 0, stream>>>(cs, Tb);
  return cudaGetLastError();
}

cudaError_t launch_vdt(const double* V, double dt, double* vdt, int n, cudaStream_t stream) {
  if (n <= 0) return cudaSuccess;
  vdt_kernel<<<(n + 255) / 256, 256, 0, stream>>>(V, dt, vdt, n);
  return cudaGetLastError();
}

cudaError_t launch_fill(double* a, size_t n, double v, cudaStream_t stream) {
  if (n == 0) return cudaSuccess;
  size_t blocks = (n + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  fill_kernel<<<(unsigned)blocks, 256, 0, stream>>>(a, n, v);
  return cudaGetLastError();
}

#ifdef LFM_CHECKED
int check_take_step(cudaStream_t s) {
  int site = 0;
  const int zero = 0;
  if (cudaMemcpyFromSymbolAsync(&site, g_check_site, sizeof(int), 0, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyToSymbolAsync(g_check_site, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyToSymbolAsync(g_check_inject, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return -1;
  return site;
}

void check_inject_step(int site, cudaStream_t s) {
  cudaMemcpyToSymbolAsync(g_check_inject, &site, sizeof(int), 0, cudaMemcpyHostToDevice, s);
  cudaStreamSynchronize(s);
}
#else
int check_take_step(cudaStream_t) { return 0; }
void check_inject_step(int, cudaStream_t) {}
#endif

}  // namespace lfm

// Face interpolation weights and the corrected laplacian's face coefficients, on the device
// (lfm_face_coeffs_device in include/lapfoam.h): the paper's "weights" loop of section "Code
// Porting" -- one thread per face, no data shared between faces -- together with the other
// per-face quantities OpenFOAM's mesh caches for the corrected laplacian (|Sf|, the
// non-orthogonal implicit coefficient, the correction vector) and the boundary faces' |Sf|
// and inverse patch-normal distance.
//
// Every product, sum, quotient and square root is rounded on its own (no contraction into
// fused multiply-adds), left to right as written, so that the results do not depend on the
// compiler's choices.
#include <cuda_runtime.h>

#include "lfm_internal.h"

namespace lfm {
namespace {

__device__ __forceinline__ double dot3(const double* a, const double* b) {
  return __dadd_rn(__dadd_rn(__dmul_rn(a[0], b[0]), __dmul_rn(a[1], b[1])), __dmul_rn(a[2], b[2]));
}

__device__ __forceinline__ void load3(const double* __restrict__ p, int64_t i, double* v) {
  v[0] = p[3 * i];
  v[1] = p[3 * i + 1];
  v[2] = p[3 * i + 2];
}

// Internal face f, owner P, neighbour N:
//   w        = |Sf.(C_N - Cf)| / (|Sf.(Cf - C_P)| + |Sf.(C_N - Cf)|)   (0.5 when that sum is
//              not above 1e-150: a degenerate face)
//   |Sf|, n  = Sf / |Sf|, d = C_N - C_P
//   delta    = 1 / max(n.d, 0.05 |d|)
//   k        = n - d delta
__global__ void face_coeffs_kernel(int32_t F, int32_t N, const int32_t* __restrict__ owner,
                                   const int32_t* __restrict__ neighbour, const double* __restrict__ Sf,
                                   const double* __restrict__ Cf, const double* __restrict__ C,
                                   double* __restrict__ w, double* __restrict__ magSf, double* __restrict__ delta,
                                   double* __restrict__ corr, int32_t* __restrict__ bad) {
  const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= F) return;
  const int P = owner[f], Q = neighbour[f];
  if ((unsigned)P >= (unsigned)N || (unsigned)Q >= (unsigned)N) {
    atomicCAS(bad, 0, 1);  // reported as LFM_EINVAL; nothing is read through a bad index
    return;
  }
  double s[3], cf[3], cp[3], cn[3], a[3], b[3], d[3], n[3];
  load3(Sf, f, s);
  load3(Cf, f, cf);
  load3(C, P, cp);
  load3(C, Q, cn);
  for (int k = 0; k < 3; ++k) {
    a[k] = __dsub_rn(cf[k], cp[k]);
    b[k] = __dsub_rn(cn[k], cf[k]);
    d[k] = __dsub_rn(cn[k], cp[k]);
  }
  const double own = fabs(dot3(s, a)), nei = fabs(dot3(s, b));
  const double tot = __dadd_rn(own, nei);
  w[f] = fabs(tot) > 1e-150 ? __ddiv_rn(nei, tot) : 0.5;
  const double mag = __dsqrt_rn(dot3(s, s));
  magSf[f] = mag;
  for (int k = 0; k < 3; ++k) n[k] = __ddiv_rn(s[k], mag);
  const double nd = fmax(dot3(n, d), __dmul_rn(0.05, __dsqrt_rn(dot3(d, d))));
  const double dl = __ddiv_rn(1.0, nd);
  delta[f] = dl;
  for (int k = 0; k < 3; ++k) corr[3 * f + k] = __dsub_rn(n[k], __dmul_rn(d[k], dl));
}

// Boundary face b of cell c: |Sf| and 1 / |n.(Cf - C_c)|.
__global__ void bface_coeffs_kernel(int32_t NB, int32_t N, const int32_t* __restrict__ bcell,
                                    const double* __restrict__ bSf, const double* __restrict__ bCf,
                                    const double* __restrict__ C, double* __restrict__ bmagSf,
                                    double* __restrict__ bdelta, int32_t* __restrict__ bad) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NB) return;
  const int c = bcell[i];
  if ((unsigned)c >= (unsigned)N) {
    atomicCAS(bad, 0, 1);
    return;
  }
  double s[3], cf[3], cc[3], n[3], t[3];
  load3(bSf, i, s);
  load3(bCf, i, cf);
  load3(C, c, cc);
  const double mag = __dsqrt_rn(dot3(s, s));
  bmagSf[i] = mag;
  for (int k = 0; k < 3; ++k) {
    n[k] = __ddiv_rn(s[k], mag);
    t[k] = __dsub_rn(cf[k], cc[k]);
  }
  bdelta[i] = __ddiv_rn(1.0, fabs(dot3(n, t)));
}

}  // namespace
}  // namespace lfm

extern "C" int lfm_face_coeffs_device(int32_t n_cells, int32_t n_faces, int32_t n_bfaces, const int32_t* owner,
                                      const int32_t* neighbour, const double* Sf, const double* Cf,
                                      const double* C, const int32_t* bface_cell, const double* bSf,
                                      const double* bCf, double* weights, double* magSf, double* deltaCoeffs,
                                      double* corr_vec, double* bmagSf, double* bdeltaCoeffs, void* stream) {
  if (n_cells < 0 || n_faces < 0 || n_bfaces < 0)
    return lfm::set_last_error(LFM_EINVAL, "lfm_face_coeffs_device: negative count");
  if (n_faces > 0 && (!owner || !neighbour || !Sf || !Cf || !C || !weights || !magSf || !deltaCoeffs || !corr_vec))
    return lfm::set_last_error(LFM_EINVAL, "lfm_face_coeffs_device: a face array is NULL");
  if (n_bfaces > 0 && (!bface_cell || !bSf || !bCf || !C || !bmagSf || !bdeltaCoeffs))
    return lfm::set_last_error(LFM_EINVAL, "lfm_face_coeffs_device: a boundary-face array is NULL");
  if (n_faces == 0 && n_bfaces == 0) return LFM_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int32_t* bad = nullptr;
  if (cudaMallocAsync(&bad, sizeof(int32_t), s) != cudaSuccess) {
    cudaGetLastError();
    return lfm::set_last_error(LFM_ECUDA, "lfm_face_coeffs_device: allocation failed");
  }
  int32_t h_bad = 0;
  cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(int32_t), s);
  if (e == cudaSuccess && n_faces > 0) {
    lfm::face_coeffs_kernel<<<(n_faces + 255) / 256, 256, 0, s>>>(n_faces, n_cells, owner, neighbour, Sf, Cf, C,
                                                                 weights, magSf, deltaCoeffs, corr_vec, bad);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && n_bfaces > 0) {
    lfm::bface_coeffs_kernel<<<(n_bfaces + 255) / 256, 256, 0, s>>>(n_bfaces, n_cells, bface_cell, bSf, bCf, C,
                                                                   bmagSf, bdeltaCoeffs, bad);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_bad, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFreeAsync(bad, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return lfm::set_last_error(LFM_ECUDA, "lfm_face_coeffs_device: %s", cudaGetErrorString(e));
  }
  if (h_bad) return lfm::set_last_error(LFM_EINVAL, "lfm_face_coeffs_device: a cell index is out of range");
  return LFM_OK;
}

// Construction of a rectilinear hexahedral box mesh in LDU form (natural numbering:
// cell c = i + nx (j + ny k)), written straight into the slot-major layout, on the device
// (lfm_upload_box) or, from the same per-cell routine, on the host (lfm_box_layout, used
// to validate the routine against the general mesh path).
//
// With natural numbering every quantity the general path derives by sorting has a closed
// form, so one thread per cell writes its row:
//   - faces are sorted by (owner, neighbour); cell c owns its +x, +y, +z faces (those that
//     exist), in that order, starting at
//       own_start(c) = (nx-1) r + i + nx (ny-1) k + nx j + [j < ny-1] i + min(c, (nz-1) nx ny)
//     with r = j + ny k (the x-, y- and z-faces owned by the cells before c);
//   - its neighbour-side faces are the +z face of c - nx ny, the +y face of c - nx and the
//     +x face of c - 1 (ascending owner, hence ascending face id);
//   - boundary faces are grouped by patch (x0, x1, y0, y1, z0, z1; x-patches ordered by
//     (k, j), y-patches by (k, i), z-patches by (j, i)); the number of boundary faces of the
//     cells before c is the sum of six closed-form counts (bstart below).
// Geometry: V = (dx dy) dz, internal |Sf| = product of the two widths in the face plane,
// deltaCoeff = 1 / (centre distance), boundary deltaCoeff = 1 / (face-to-centre distance).
#include <cmath>

#include <cuda_runtime.h>

#include "lfm_internal.h"

namespace lfm {
namespace {

struct BoxDims {
  long long nx, ny, nz;
  int W;
  const double *xs, *ys, *zs;
};

struct BoxOut {
  int32_t *slot_other, *slot_face;
  uint32_t* face_slots;
  double *V, *magSf, *delta;
  int32_t *b_start, *b_face, *bcell;
  double *bmagSf, *bdelta;
};

__host__ __device__ inline long long box_own_start(const BoxDims& d, long long i, long long j, long long k) {
  const long long nx = d.nx, ny = d.ny, nz = d.nz;
  const long long c = i + nx * (j + ny * k);
  const long long r = j + ny * k;
  const long long fx = (nx - 1) * r + i;
  const long long fy = nx * (ny - 1) * k + nx * j + (j < ny - 1 ? i : 0);
  const long long lim = (nz - 1) * nx * ny;
  const long long fz = c < lim ? c : lim;
  return fx + fy + fz;
}

__host__ __device__ inline long long box_bstart(const BoxDims& d, long long i, long long j, long long k) {
  const long long nx = d.nx, ny = d.ny, nz = d.nz;
  const long long c = i + nx * (j + ny * k);
  const long long r = j + ny * k;
  const long long ax0 = r + (i > 0 ? 1 : 0);       // cells before c with i = 0
  const long long ax1 = r;                         // ... with i = nx-1
  const long long ay0 = nx * k + (j > 0 ? nx : i);  // ... with j = 0
  const long long ay1 = nx * k + (j == ny - 1 ? i : 0);
  const long long az0 = k > 0 ? nx * ny : c;        // ... with k = 0
  const long long az1 = k == nz - 1 ? c - (nz - 1) * nx * ny : 0;
  return ax0 + ax1 + ay0 + ay1 + az0 + az1;
}

__host__ __device__ inline double box_centre(const double* v, long long i) { return 0.5 * (v[i] + v[i + 1]); }
__host__ __device__ inline double box_width(const double* v, long long i) { return v[i + 1] - v[i]; }

// Writes everything that belongs to cell c (c == N writes the final boundary start).
__host__ __device__ inline void box_cell(const BoxDims& d, long long c, const BoxOut& o) {
  const long long nx = d.nx, ny = d.ny, nz = d.nz;
  const long long N = nx * ny * nz;
  if (c == N) {
    o.b_start[N] = (int32_t)(2 * (ny * nz + nx * nz + nx * ny));
    return;
  }
  const long long i = c % nx, j = (c / nx) % ny, k = c / (nx * ny);
  const double hx = box_width(d.xs, i), hy = box_width(d.ys, j), hz = box_width(d.zs, k);
  o.V[c] = (hx * hy) * hz;

  int s = 0;
  if (k > 0) {
    o.slot_other[(size_t)s * N + c] = (int32_t)(c - nx * ny);
    o.slot_face[(size_t)s * N + c] = (int32_t)(box_own_start(d, i, j, k - 1) + (i < nx - 1) + (j < ny - 1));
    ++s;
  }
  if (j > 0) {
    o.slot_other[(size_t)s * N + c] = (int32_t)(c - nx);
    o.slot_face[(size_t)s * N + c] = (int32_t)(box_own_start(d, i, j - 1, k) + (i < nx - 1));
    ++s;
  }
  if (i > 0) {
    o.slot_other[(size_t)s * N + c] = (int32_t)(c - 1);
    o.slot_face[(size_t)s * N + c] = (int32_t)box_own_start(d, i - 1, j, k);
    ++s;
  }
  // an owned face sits in the neighbour's row after the neighbour's lower-ordered faces:
  // +x: after its z- and y-faces, +y: after its z-face, +z: first
  const long long mate_x = (k > 0) + (j > 0), mate_y = (k > 0), mate_z = 0;
  long long f = box_own_start(d, i, j, k);
  if (i < nx - 1) {
    o.magSf[f] = hy * hz;
    o.delta[f] = 1.0 / (box_centre(d.xs, i + 1) - box_centre(d.xs, i));
    o.slot_other[(size_t)s * N + c] = (int32_t)(c + 1);
    o.slot_face[(size_t)s * N + c] = (int32_t)f;
    o.face_slots[2 * f] = (uint32_t)(s * N + c);
    o.face_slots[2 * f + 1] = (uint32_t)(mate_x * N + c + 1);
    ++f;
    ++s;
  }
  if (j < ny - 1) {
    o.magSf[f] = hx * hz;
    o.delta[f] = 1.0 / (box_centre(d.ys, j + 1) - box_centre(d.ys, j));
    o.slot_other[(size_t)s * N + c] = (int32_t)(c + nx);
    o.slot_face[(size_t)s * N + c] = (int32_t)f;
    o.face_slots[2 * f] = (uint32_t)(s * N + c);
    o.face_slots[2 * f + 1] = (uint32_t)(mate_y * N + c + nx);
    ++f;
    ++s;
  }
  if (k < nz - 1) {
    o.magSf[f] = hx * hy;
    o.delta[f] = 1.0 / (box_centre(d.zs, k + 1) - box_centre(d.zs, k));
    o.slot_other[(size_t)s * N + c] = (int32_t)(c + nx * ny);
    o.slot_face[(size_t)s * N + c] = (int32_t)f;
    o.face_slots[2 * f] = (uint32_t)(s * N + c);
    o.face_slots[2 * f + 1] = (uint32_t)(mate_z * N + c + nx * ny);
    ++f;
    ++s;
  }
  for (; s < d.W; ++s) {
    o.slot_other[(size_t)s * N + c] = (int32_t)c;
    o.slot_face[(size_t)s * N + c] = -1;
  }

  long long at = box_bstart(d, i, j, k);
  o.b_start[c] = (int32_t)at;
  const long long px1 = ny * nz, py0 = 2 * ny * nz, py1 = py0 + nx * nz, pz0 = py1 + nx * nz, pz1 = pz0 + nx * ny;
  double bd[6];
  long long bb[6];
  double ba[6];
  int nb = 0;
  if (i == 0) { bb[nb] = k * ny + j; ba[nb] = hy * hz; bd[nb] = 1.0 / fabs(d.xs[0] - box_centre(d.xs, i)); ++nb; }
  if (i == nx - 1) { bb[nb] = px1 + k * ny + j; ba[nb] = hy * hz; bd[nb] = 1.0 / fabs(d.xs[nx] - box_centre(d.xs, i)); ++nb; }
  if (j == 0) { bb[nb] = py0 + k * nx + i; ba[nb] = hx * hz; bd[nb] = 1.0 / fabs(d.ys[0] - box_centre(d.ys, j)); ++nb; }
  if (j == ny - 1) { bb[nb] = py1 + k * nx + i; ba[nb] = hx * hz; bd[nb] = 1.0 / fabs(d.ys[ny] - box_centre(d.ys, j)); ++nb; }
  if (k == 0) { bb[nb] = pz0 + j * nx + i; ba[nb] = hx * hy; bd[nb] = 1.0 / fabs(d.zs[0] - box_centre(d.zs, k)); ++nb; }
  if (k == nz - 1) { bb[nb] = pz1 + j * nx + i; ba[nb] = hx * hy; bd[nb] = 1.0 / fabs(d.zs[nz] - box_centre(d.zs, k)); ++nb; }
  for (int q = 0; q < nb; ++q) {
    o.b_face[at++] = (int32_t)bb[q];
    o.bcell[bb[q]] = (int32_t)c;
    o.bmagSf[bb[q]] = ba[q];
    o.bdelta[bb[q]] = bd[q];
  }
}

__global__ void box_kernel(BoxDims d, BoxOut o) {
  const long long N = d.nx * d.ny * d.nz;
  const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (c <= N) box_cell(d, c, o);
}

}  // namespace

int box_slot_width(long long nx, long long ny, long long nz) {
  auto w = [](long long n) { return n >= 3 ? 2 : (n == 2 ? 1 : 0); };
  return w(nx) + w(ny) + w(nz);
}

cudaError_t launch_box(long long nx, long long ny, long long nz, int W, const double* xs, const double* ys,
                       const double* zs, const CaseDev& cs, cudaStream_t stream) {
  BoxDims d{nx, ny, nz, W, xs, ys, zs};
  BoxOut o{const_cast<int32_t*>(cs.slot_other), const_cast<int32_t*>(cs.slot_face),
           const_cast<uint32_t*>(cs.face_slots), const_cast<double*>(cs.V),
           const_cast<double*>(cs.magSf), const_cast<double*>(cs.delta), const_cast<int32_t*>(cs.b_start),
           const_cast<int32_t*>(cs.b_face), const_cast<int32_t*>(cs.bcell), const_cast<double*>(cs.bmagSf),
           const_cast<double*>(cs.bdelta)};
  const long long threads = nx * ny * nz + 1;
  box_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, stream>>>(d, o);
  return cudaGetLastError();
}

void box_layout_host(long long nx, long long ny, long long nz, int W, const double* xs, const double* ys,
                     const double* zs, int32_t* slot_other, int32_t* slot_face, uint32_t* face_slots, double* V,
                     double* magSf, double* delta, int32_t* b_start, int32_t* b_face, int32_t* bcell,
                     double* bmagSf, double* bdelta) {
  BoxDims d{nx, ny, nz, W, xs, ys, zs};
  BoxOut o{slot_other, slot_face, face_slots, V, magSf, delta, b_start, b_face, bcell, bmagSf, bdelta};
  const long long N = nx * ny * nz;
  for (long long c = 0; c <= N; ++c) box_cell(d, c, o);
}

}  // namespace lfm

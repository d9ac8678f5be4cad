// Face-to-cell addressing of a general LDU mesh built on the device (the paper's section
// "Code Porting": the lists of lists ownerStart/ownerList, neighbourStart/neighbourList and
// the per-patch face lists are built once per mesh with parallel sort, reduce and scan).
//
// From owner[F], neighbour[F] (faces in upper-triangular order) and bface_cell[NB]:
//   - owner-side faces of cell c: [lower_bound(owner, c), lower_bound(owner, c + 1)) -- the
//     faces are sorted by owner, so a binary search replaces the paper's sort + reduce;
//   - neighbour-side faces: a counting sort by neighbour -- counts by atomic increments
//     (exact, order-free), exclusive scan into lo_start, placement by atomic slot claims, then
//     each cell's short list sorted by face id, so the result is the unique ascending order
//     (deterministic, equal to the host's stable counting sort);
//   - boundary faces of each cell the same way (b_start, b_face);
//   - the slot-major rows (slot_other, slot_face: neighbour-side faces, owned faces, padding)
//     and each face's two slot positions (face_slots).
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "lfm_internal.h"

namespace lfm {
namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int64_t kScanBlock = (int64_t)kScanThreads * kScanItems;

__global__ void count_kernel(const int32_t* __restrict__ key, int64_t n, int32_t* __restrict__ cnt) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) atomicAdd(cnt + key[i], 1);
}

// Exclusive scan of one block of kScanBlock items (out[i] = sum of in[block start .. i));
// the block's total goes to sums[blockIdx.x].
__global__ void __launch_bounds__(kScanThreads) scan_block_kernel(const int32_t* __restrict__ in, int64_t n,
                                                                  int32_t* __restrict__ out,
                                                                  int32_t* __restrict__ sums) {
  __shared__ int32_t warp_tot[kScanThreads / 32];
  const int64_t base = blockIdx.x * kScanBlock + (int64_t)threadIdx.x * kScanItems;
  int32_t v[kScanItems];
  int32_t t = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = base + k < n ? in[base + k] : 0;
    t += v[k];
  }
  // inclusive scan of the thread totals within the warp, then across warps
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t inc = t;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) warp_tot[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    int32_t w = lane < kScanThreads / 32 ? warp_tot[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < kScanThreads / 32) warp_tot[lane] = w;  // inclusive over warps
  }
  __syncthreads();
  int32_t run = inc - t + (warp > 0 ? warp_tot[warp - 1] : 0);  // exclusive prefix of this thread
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
  if (threadIdx.x == kScanThreads - 1) sums[blockIdx.x] = warp_tot[kScanThreads / 32 - 1];
}

__global__ void scan_add_kernel(int32_t* __restrict__ out, int64_t n, const int32_t* __restrict__ offsets) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] += offsets[i / kScanBlock];
}

__global__ void set_value_kernel(int32_t* __restrict__ p, const int32_t* __restrict__ src, int32_t v) {
  *p = src ? *src : v;
}

__global__ void place_kernel(const int32_t* __restrict__ key, int64_t n, const int32_t* __restrict__ start,
                             int32_t* __restrict__ fill, int32_t* __restrict__ order) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) {
    const int32_t k = key[i];
    order[start[k] + atomicAdd(fill + k, 1)] = (int32_t)i;
  }
}

// Sorts each segment order[start[c] .. start[c+1]) ascending (segments are short: the
// faces of one cell).
__global__ void sort_segments_kernel(const int32_t* __restrict__ start, int32_t n_keys, int32_t* __restrict__ order) {
  const int32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_keys) return;
  const int32_t a = start[c], b = start[c + 1];
  for (int32_t i = a + 1; i < b; ++i) {
    const int32_t v = order[i];
    int32_t j = i - 1;
    while (j >= a && order[j] > v) {
      order[j + 1] = order[j];
      --j;
    }
    order[j + 1] = v;
  }
}

__device__ __forceinline__ int32_t lower_bound(const int32_t* __restrict__ a, int32_t n, int32_t v) {
  int32_t lo = 0, hi = n;
  while (lo < hi) {
    const int32_t mid = lo + ((hi - lo) >> 1);
    if (a[mid] < v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__global__ void slots_kernel(int32_t N, int32_t F, int32_t W, const int32_t* __restrict__ owner,
                             const int32_t* __restrict__ neighbour, const int32_t* __restrict__ lo_start,
                             const int32_t* __restrict__ losort, int32_t* __restrict__ slot_other,
                             int32_t* __restrict__ slot_face, uint32_t* __restrict__ face_slots) {
  const int32_t c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N) return;
  const size_t n = (size_t)N;
  int k = 0;
  for (int32_t i = lo_start[c]; i < lo_start[c + 1]; ++i, ++k) {
    const int32_t f = losort[i];
    const size_t at = (size_t)k * n + c;
    slot_other[at] = owner[f];
    slot_face[at] = f;
    face_slots[2 * (size_t)f + 1] = (uint32_t)at;
  }
  const int32_t f0 = lower_bound(owner, F, c), f1 = lower_bound(owner, F, c + 1);
  for (int32_t f = f0; f < f1; ++f, ++k) {
    const size_t at = (size_t)k * n + c;
    slot_other[at] = neighbour[f];
    slot_face[at] = f;
    face_slots[2 * (size_t)f] = (uint32_t)at;
  }
  for (; k < W; ++k) {
    const size_t at = (size_t)k * n + c;
    slot_other[at] = c;
    slot_face[at] = -1;
  }
}

unsigned grid(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// out[0 .. n] = exclusive scan of in[0 .. n), out[n] the total. tmp: scratch of
// scan_tmp_ints(n) ints.
cudaError_t exclusive_scan(const int32_t* in, int32_t* out, int64_t n, int32_t* tmp, cudaStream_t s) {
  if (n == 0) {
    set_value_kernel<<<1, 1, 0, s>>>(out, nullptr, 0);
    return cudaGetLastError();
  }
  const int64_t nb = (n + kScanBlock - 1) / kScanBlock;
  int32_t* sums = tmp;            // [nb]
  int32_t* sums_scan = tmp + nb;  // [nb + 1]
  scan_block_kernel<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, out, sums);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (nb == 1) {
    set_value_kernel<<<1, 1, 0, s>>>(out + n, sums, 0);
    return cudaGetLastError();
  }
  if ((e = exclusive_scan(sums, sums_scan, nb, tmp + 2 * nb + 1, s)) != cudaSuccess) return e;
  scan_add_kernel<<<grid(n, 256), 256, 0, s>>>(out, n, sums_scan);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  set_value_kernel<<<1, 1, 0, s>>>(out + n, sums_scan + nb, 0);
  return cudaGetLastError();
}

int64_t scan_tmp_ints(int64_t n) {
  int64_t total = 0;
  while (n > 1) {
    const int64_t nb = (n + kScanBlock - 1) / kScanBlock;
    total += 2 * nb + 1;
    if (nb == 1) break;
    n = nb;
  }
  return total + 8;
}

}  // namespace

cudaError_t build_addressing(int32_t N, int32_t F, int32_t NB, int32_t W, const int32_t* owner,
                             const int32_t* neighbour, const int32_t* bface_cell, int32_t* slot_other,
                             int32_t* slot_face, uint32_t* face_slots, int32_t* b_start, int32_t* b_face,
                             cudaStream_t s) {
  // scratch: counts / fill [N], lo_start [N+1], losort [F], scan temporaries
  const int64_t tmp_ints = scan_tmp_ints(N);
  const size_t ints = (size_t)N + (size_t)(N + 1) + (size_t)(F > 0 ? F : 1) + (size_t)tmp_ints;
  int32_t* buf = nullptr;
  cudaError_t e = cudaMallocAsync(&buf, sizeof(int32_t) * ints, s);
  if (e != cudaSuccess) return e;
  int32_t* cnt = buf;
  int32_t* lo_start = cnt + N;
  int32_t* losort = lo_start + (N + 1);
  int32_t* tmp = losort + (F > 0 ? F : 1);
  do {
    // neighbour-side lists
    if ((e = cudaMemsetAsync(cnt, 0, sizeof(int32_t) * N, s)) != cudaSuccess) break;
    if (F > 0) count_kernel<<<grid(F, 256), 256, 0, s>>>(neighbour, F, cnt);
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    if ((e = exclusive_scan(cnt, lo_start, N, tmp, s)) != cudaSuccess) break;
    if ((e = cudaMemsetAsync(cnt, 0, sizeof(int32_t) * N, s)) != cudaSuccess) break;
    if (F > 0) place_kernel<<<grid(F, 256), 256, 0, s>>>(neighbour, F, lo_start, cnt, losort);
    sort_segments_kernel<<<grid(N, 256), 256, 0, s>>>(lo_start, N, losort);
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    // boundary faces per cell
    if ((e = cudaMemsetAsync(cnt, 0, sizeof(int32_t) * N, s)) != cudaSuccess) break;
    if (NB > 0) count_kernel<<<grid(NB, 256), 256, 0, s>>>(bface_cell, NB, cnt);
    if ((e = cudaGetLastError()) != cudaSuccess) break;
    if ((e = exclusive_scan(cnt, b_start, N, tmp, s)) != cudaSuccess) break;
    if ((e = cudaMemsetAsync(cnt, 0, sizeof(int32_t) * N, s)) != cudaSuccess) break;
    if (NB > 0) place_kernel<<<grid(NB, 256), 256, 0, s>>>(bface_cell, NB, b_start, cnt, b_face);
    sort_segments_kernel<<<grid(N, 256), 256, 0, s>>>(b_start, N, b_face);
    // slot rows and face slot positions
    slots_kernel<<<grid(N, 256), 256, 0, s>>>(N, F, W, owner, neighbour, lo_start, losort, slot_other, slot_face,
                                               face_slots);
    e = cudaGetLastError();
  } while (false);
  cudaError_t e2 = cudaFreeAsync(buf, s);
  return e != cudaSuccess ? e : e2;
}

}  // namespace lfm

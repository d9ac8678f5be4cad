// Device primitives: bounded team barriers with deterministic reductions.
//
// A "team" is a set of co-resident CTAs (a cooperative launch guarantees co-residency)
// working on one case. Each barrier may carry up to kMaxSums FP64 sums: every CTA reduces
// its threads' values with a fixed warp-shuffle / shared-memory tree, writes the CTA total
// to its slot of a partial table, and arrives on a counter. The last CTA to arrive adds the
// slots in rank order (lane l takes ranks l, l+32, ...; then a fixed xor tree), publishes
// the sums and releases the barrier by bumping a generation word. The result depends only
// on the team size, never on arrival order, so repeated runs are bitwise identical. The
// barrier is a chain of L2 round trips, so it is built to keep that chain short: arrival is
// one acquire-release atomic, the release one release store, and no fence sits on the
// critical path (about 5.4 us with one sum for 304 CTAs on GB300, 7.7 us with a fence before
// the arrival and around the last arriver's reduction). Each further sum costs more than a
// round trip does: the CTA's own reduction adds in FP64, which GB300 issues slowly, so
// block_reduce keeps its FP64 adds few.
//
// Every wait is bounded: a waiter that sees no release within the launch's time limit (or
// sees another CTA's error) records an error status and the caller leaves the kernel.
#pragma once

#include <cstdint>

#include "lfm_internal.h"

namespace lfm {

__device__ __forceinline__ uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int ld_volatile_i32(const int32_t* p) {
  return *reinterpret_cast<const volatile int32_t*>(p);
}

// ---- checked builds ----------------------------------------------------------------------
// Compiled with -DLFM_CHECKED (the library variant liblapfoam_checked.so), every index a
// kernel reads from the mesh's addressing and then uses as an address (a slot's neighbour
// cell, a face's slot positions, a boundary face) is tested against its array's extent
// first. A bad index is replaced by an in-range one (the caller's fallback), and the first
// failing site is recorded in a word of this translation unit, which the host reads after
// the launch and reports as LFM_EINVAL. Nothing reads out of bounds and nothing traps: the
// team barriers keep working and the context stays usable. In the normal build the checks
// compile to nothing. check_inject (a test hook) makes one site report as failing without
// any bad index.
enum CheckSite {
  kChkSlotCell = 1,   // a slot's neighbour cell (FP64 / FP32 passes, set-up)
  kChkFaceSlot = 2,   // face <-> slot addressing: a face's slot positions, a slot's face
  kChkBFace = 3,      // boundary addressing: a cell's boundary faces, a boundary face's cell
  kChkSlotCellDf = 4  // a slot's neighbour cell (df64 passes)
};
#ifdef LFM_CHECKED
namespace {
__device__ int g_check_site;    // first failing site, 0 while none
__device__ int g_check_inject;  // test hook: this site reports as failing
}  // namespace
__device__ __forceinline__ int checked_index(int i, int n, int fallback, int site) {
  const bool bad = (unsigned)i >= (unsigned)n;
  if (bad || g_check_inject == site) atomicCAS(&g_check_site, 0, site);
  return bad ? fallback : i;
}
#define LFM_IDX(i, n, fallback, site) ::lfm::checked_index((int)(i), (int)(n), (fallback), (site))
#else
#define LFM_IDX(i, n, fallback, site) (i)
#endif

struct Team {
  int size;
  int rank;
  SyncWords* sw;
  double* partials;
  uint64_t timeout_ns;
};

// Shared scratch a CTA needs for team_allreduce.
constexpr int kRedSlots = 256;  // block_reduce's shared partial sums (all NS sums together)

struct TeamShared {
  double red[kRedSlots];
  double out[kMaxSums];
  int flag[4];
  unsigned gen;  // thread 0: the team's generation before this CTA's next arrival
};

// Thread 0 of a CTA, when the CTA joins a team (before its first arrival): the team's
// generation word, which no barrier can move before this CTA has arrived. team_allreduce
// then tracks the generation itself (one more per barrier passed), so that no load of it
// sits before an arrival.
__device__ __forceinline__ void team_join(const Team& tm, TeamShared& sh) {
  sh.gen = *reinterpret_cast<volatile unsigned*>(&tm.sw->gen);
}

// Spins until *gen != g. False (with the error recorded) when the time limit runs out or
// another CTA has recorded an error. The load is an acquire: what the releasing CTA wrote
// before its release is visible to this thread afterwards, without a further fence.
__device__ __forceinline__ bool wait_generation(unsigned* gen, unsigned g, int32_t* status,
                                                uint64_t timeout_ns) {
  uint64_t t0 = global_timer_ns();
  unsigned spins = 0;
  while (ld_acquire_u32(gen) == g) {
    ++spins;
    if (spins > 16) __nanosleep(32);
    if ((spins & 31u) == 0) {
      if (ld_volatile_i32(status) != 0) return false;
      if (global_timer_ns() - t0 > timeout_ns) {
        atomicCAS(status, 0, (int32_t)LFM_ETIMEOUT);
        return false;
      }
    }
  }
  return true;
}

// Arrival at a team barrier: one acquire-release add on the arrival counter (the release
// orders this CTA's partial sums before it, the acquire makes every earlier arrival's
// partial sums visible to the last arriver).
__device__ __forceinline__ unsigned arrive_acq_rel(unsigned* count) {
  unsigned old;
  asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], 1;" : "=r"(old) : "l"(count) : "memory");
  return old;
}

// Fixed-pattern reduction of NS values over the CTA: each warp folds its lanes by an xor tree
// down to vpw partial sums (lanes 0 .. vpw - 1; vpw the largest of 8, 4, 2, 1 whose partials
// of 32 warps and all sums fit kRedSlots), the partials go through shared memory, and warp 0
// sums them: lane l takes partials l, l + 32, ... in index order, then a five-level xor
// tree. Totals land in sh.out (visible after the caller's next __syncthreads). The order
// depends only on the block size. The FP64 pipe issues about two operations per clock per
// SM on GB300, so the fewer FP64 adds matter: against a full xor tree in every warp this
// measured 5.95 -> 5.45, 9.34 -> 7.63 and 15.17 -> 12.90 us per barrier with 1, 2 and 4
// sums over 304 CTAs.
template <int NS>
__host__ __device__ constexpr int partials_per_warp() {  // sized for the largest block, 32 warps
  return 32 * 8 * NS <= kRedSlots ? 8 : 32 * 4 * NS <= kRedSlots ? 4 : 32 * 2 * NS <= kRedSlots ? 2 : 1;
}

template <int NS>
__device__ __forceinline__ void block_reduce(double* v, TeamShared& sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  constexpr int vpw = partials_per_warp<NS>();
#pragma unroll
  for (int k = 0; k < NS; ++k) {
#pragma unroll
    for (int o = 16; o >= vpw; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
  }
  const int nv = nw * vpw;
  if (lane < vpw) {
#pragma unroll
    for (int k = 0; k < NS; ++k) sh.red[k * nv + warp * vpw + lane] = v[k];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      double t = 0.0;
      for (int i = lane; i < nv; i += 32) t += sh.red[k * nv + i];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (lane == 0) sh.out[k] = t;
    }
  }
}

// Team-wide barrier carrying NS sums. On return (true) v[k] holds the team totals in every
// thread. False: a wait ran out or another CTA failed; the caller must leave the kernel.
// Protocol: thread 0 stores the CTA's partial sums and arrives (one acquire-release add;
// the generation it waits on is its own count, see team_join); the CTA that finds size - 1 arrivals before its own is the last:
// warp 0 loads all partial sums at once, adds them in rank order (lane l takes ranks l,
// l + 32, ..., then a fixed xor tree), publishes the totals, clears the counter and releases
// the generation with a release store (which orders the totals and the cleared counter
// before it). The others wait for the generation with acquire loads and then read the
// totals. The sums depend only on the team size, never on arrival order. (Detecting the
// last arrival by a remainder modulo the team size, with a counter never cleared, measured
// 10 % slower in the mixed form's A p: the division's code sits in its inner loop.)
template <int NS>
__device__ bool team_allreduce(const Team& tm, double* v, TeamShared& sh) {
  // Every thread's global writes of the phase must be ordered before thread 0 signals
  // arrival: block_reduce synchronises the CTA itself; a barrier without sums needs its own.
  if constexpr (NS > 0) {
    block_reduce<NS>(v, sh);
  } else {
    __syncthreads();
  }
  if (tm.size == 1) {
    __syncthreads();
    if constexpr (NS > 0) {
#pragma unroll
      for (int k = 0; k < NS; ++k) v[k] = sh.out[k];
    }
    return true;
  }
  if (threadIdx.x == 0) {
    if constexpr (NS > 0) {
#pragma unroll
      for (int k = 0; k < NS; ++k) __stcg(&tm.partials[tm.rank * kMaxSums + k], sh.out[k]);
    }
    const unsigned g = sh.gen;
    const unsigned prev = arrive_acq_rel(&tm.sw->count);
    const int last = prev == (unsigned)(tm.size - 1);
    int ok = 1;
    if (!last) {
      ok = wait_generation(&tm.sw->gen, g, &tm.sw->status, tm.timeout_ns);
      if constexpr (NS > 0) {
        if (ok) {
#pragma unroll
          for (int k = 0; k < NS; ++k) sh.out[k] = __ldcg(&tm.sw->scalars[k]);
        }
      }
    }
    sh.flag[0] = last;
    sh.flag[1] = ok;
    sh.flag[2] = (int)g;
    sh.gen = g + 1u;
  }
  __syncthreads();
  if (!sh.flag[1]) return false;
  if (sh.flag[0]) {
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      if constexpr (NS > 0) {
        // loads first, 16 values per lane in flight (lane l takes ranks l, l + 32, ...), then
        // the adds; 16 doubles per lane keep within the kernels' 64-register budget
        constexpr int kBatch = 16 / NS;
        double t[NS];
#pragma unroll
        for (int k = 0; k < NS; ++k) t[k] = 0.0;
        for (int r0 = 0; r0 < tm.size; r0 += 32 * kBatch) {
          double buf[kBatch][NS];
#pragma unroll
          for (int i = 0; i < kBatch; ++i) {
            const int r = r0 + lane + 32 * i;
#pragma unroll
            for (int k = 0; k < NS; ++k) buf[i][k] = r < tm.size ? __ldcg(&tm.partials[r * kMaxSums + k]) : 0.0;
          }
#pragma unroll
          for (int i = 0; i < kBatch; ++i)
#pragma unroll
            for (int k = 0; k < NS; ++k) t[k] += buf[i][k];
        }
#pragma unroll
        for (int k = 0; k < NS; ++k) {
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) t[k] += __shfl_xor_sync(0xffffffffu, t[k], o);
        }
        if (lane == 0) {
#pragma unroll
          for (int k = 0; k < NS; ++k) {
            sh.out[k] = t[k];
            __stcg(&tm.sw->scalars[k], t[k]);
          }
        }
      }
      __syncwarp();
      if (lane == 0) {
        tm.sw->count = 0u;  // ordered before the release below; no CTA arrives again before it
        st_release_u32(&tm.sw->gen, (unsigned)sh.flag[2] + 1u);
      }
    }
    __syncthreads();
  }
  if constexpr (NS > 0) {
#pragma unroll
    for (int k = 0; k < NS; ++k) v[k] = sh.out[k];
  }
  return true;
}

// Team-wide barrier without sums.
__device__ __forceinline__ bool team_barrier(const Team& tm, TeamShared& sh) {
  return team_allreduce<0>(tm, nullptr, sh);
}

// ---- bulk copies global -> shared, completed on an mbarrier ------------------------------
// One thread arms a stage's mbarrier with the byte count it expects and issues the bulk
// copies (cp.async.bulk: the copy engine moves the bytes, no thread registers hold them);
// every thread then waits on the barrier's phase. Source and destination must be 16-byte
// aligned and each size a multiple of 16 bytes.
extern __shared__ __align__(128) unsigned char lfm_dyn_smem[];

namespace {
// Test hook (set by the host for one launch): this CTA issues no copy for its first staged
// tile, so that its bounded wait runs out (-1: none).
__device__ int g_skip_copy_cta = -1;
}  // namespace

__device__ __forceinline__ unsigned dyn_smem_bytes() {
  unsigned v;
  asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(v));
  return v;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Makes the initialised barriers visible to the copy engine (the async proxy).
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// L2 policy for data read once per pass (the matrix): evicted first, so that it does not
// displace the gathered vector.
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar, uint64_t pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(pol)
      : "memory");
}

// Waits for the barrier's phase with the given parity. False (with LFM_ETIMEOUT recorded,
// unless another error was) when the launch's time limit runs out or another CTA has
// recorded an error.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, int32_t* status, uint64_t timeout_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_timer_ns();
  for (unsigned spins = 1;; ++spins) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((spins & 15u) == 0) {
      if (ld_volatile_i32(status) != 0) return false;
      if (global_timer_ns() - t0 > timeout_ns) {
        atomicCAS(status, 0, (int32_t)LFM_ETIMEOUT);
        return false;
      }
    }
  }
}

// Waits for the barrier's phase without regard to the launch's status (bounded by the time
// limit): the drain of copies still in flight before a CTA that failed leaves.
__device__ __forceinline__ void mbar_drain(uint64_t* bar, unsigned parity, uint64_t timeout_ns) {
  const uint64_t t0 = global_timer_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (global_timer_ns() - t0 > timeout_ns) return;
  }
}

// Runs body over the CTA's cells [c0, c1) in tiles of TC cells whose per-cell rows arrive in
// shared memory by bulk copies, two stages of kStage bytes at the start of the dynamic shared
// memory (their mbarriers after them). issue(stage, t0, n, bar, pol), called by thread 0
// only, arms bar with the tile's byte count and issues its copies into stage; body(stage, t0,
// nt) processes tile [t0, t0 + nt) once its copies have landed. The copy of tile t + 2 is
// issued as soon as every thread is done with tile t. False when a wait ran out or another CTA
// failed (status recorded): the CTA then lets its copies in flight land (bounded) before the
// caller leaves.
template <int TC, unsigned kStage, typename Issue, typename Body>
__device__ __forceinline__ bool staged_tiles(int c0, int c1, const Team& tm, Issue&& issue, Body&& body) {
  unsigned char* sm = lfm_dyn_smem;
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + 2 * kStage);
  const int tid = threadIdx.x;
  const int ntiles = c1 > c0 ? (c1 - c0 + TC - 1) / TC : 0;
  if (tid == 0) {
    mbar_init(bar, 1);
    mbar_init(bar + 1, 1);
    mbar_init_fence();
    const uint64_t pol = l2_evict_first_policy();
    for (int t = 0; t < 2 && t < ntiles; ++t) {
      const int t0 = c0 + t * TC;
      if (t == 0 && (int)blockIdx.x == g_skip_copy_cta) continue;
      issue(sm + (t & 1) * kStage, t0, min(TC, c1 - t0), bar + (t & 1), pol);
    }
  }
  __syncthreads();
  int t = 0;
  bool failed = false;
  for (; t < ntiles; ++t) {
    const int s = t & 1;
    const bool got = mbar_wait(bar + s, (t >> 1) & 1, &tm.sw->status, tm.timeout_ns);
    const int t0 = c0 + t * TC;
    if (got) body(static_cast<const unsigned char*>(sm + s * kStage), t0, min(TC, c1 - t0));
    if (__syncthreads_or(!got)) {  // every thread is done with stage s (or one wait failed)
      failed = true;
      break;
    }
    if (tid == 0 && t + 2 < ntiles) {
      const int t2 = t0 + 2 * TC;
      issue(sm + s * kStage, t2, min(TC, c1 - t2), bar + s, l2_evict_first_policy());
    }
  }
  if (tid == 0) {
    if (failed)
      for (int u = t; u < ntiles && u < t + 2; ++u) mbar_drain(bar + (u & 1), (u >> 1) & 1, tm.timeout_ns);
    mbar_inval(bar);
    mbar_inval(bar + 1);
    if (!failed && tm.rank == 0) ++tm.sw->staged;  // read back by the host (a test's evidence)
  }
  __syncthreads();
  return !failed;
}

// Records an error status for the launch (first error wins).
__device__ __forceinline__ void set_status(SyncWords* sw, int32_t code) {
  atomicCAS(&sw->status, 0, code);
}

}  // namespace lfm

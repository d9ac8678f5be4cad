// Batched form: many independent cases in one persistent cooperative launch.
//
// The host turns the member cases into jobs: case c needs a team of k_c CTAs (from its
// size), and job j owns tickets [job_start[j], job_start[j+1]). Jobs are ordered longest
// first. Every CTA of the launch loops: take the next ticket (one atomicAdd), find its job
// and its rank in the job's team by binary search over job_start, copy the case descriptor
// to shared memory and run the case's steps with the case's own team barriers and partial
// sums, then take another ticket. Tickets are handed out in increasing order, so at any
// time at most one job -- the one whose tickets are being handed out -- can have members
// waiting for team-mates; every other busy CTA belongs to a fully staffed job and will come
// back for a ticket, so each job is staffed in finite time (no deadlock, given k_c <= CTAs).
#include <cuda_runtime.h>

#include "lfm_device.cuh"
#include "lfm_internal.h"
#include "lfm_solve.cuh"
#include "lfm_solve_df.cuh"
#include "lfm_solve_mixed_df.cuh"

namespace lfm {
namespace {

template <int B, int W, int kForm>
__global__ void __launch_bounds__(B, 1024 / B) batch_kernel(const CaseDev* __restrict__ cases,
                                                  const int32_t* __restrict__ job_case,
                                                  const int32_t* __restrict__ job_start, BatchHeader* hdr,
                                                  int32_t* __restrict__ case_step,
                                                  const int32_t* __restrict__ case_cap, Launch L, int n_steps) {
  __shared__ TeamShared sh;
  __shared__ CaseDev s_cs;
  __shared__ int s_job[4];
  const int n_jobs = hdr->n_jobs, n_tickets = hdr->n_tickets;
  for (;;) {
    if (threadIdx.x == 0) {
      const int t = atomicAdd(&hdr->ticket, 1);
      int c = -1, rank = 0, size = 0;
      if (t < n_tickets && n_jobs > 0) {
        int lo = 0, hi = n_jobs - 1;  // largest j with job_start[j] <= t
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (job_start[mid] <= t) lo = mid; else hi = mid - 1;
        }
        c = job_case[lo];
        rank = t - job_start[lo];
        size = job_start[lo + 1] - job_start[lo];
      }
      s_job[0] = c;
      s_job[1] = rank;
      s_job[2] = size;
    }
    __syncthreads();
    const int c = s_job[0];
    if (c < 0) break;
    {
      const int* src = reinterpret_cast<const int*>(cases + c);
      int* dst = reinterpret_cast<int*>(&s_cs);
      for (int i = threadIdx.x; i < (int)(sizeof(CaseDev) / sizeof(int)); i += B) dst[i] = src[i];
    }
    __syncthreads();
    const Team tm{s_job[2], s_job[1], s_cs.sync, s_cs.partials, L.timeout_ns};
    if (threadIdx.x == 0) team_join(tm, sh);
    const int base = case_step[c];
    // a case whose cap is reached runs no step; its team's CTAs go back for tickets at once
    const int run = min(n_steps, case_cap[c] - base);
    if (run > 0) {
      if constexpr (kForm == kBatchFp64) {
        run_steps_f64<B, W>(s_cs, s_cs, tm, run, kModeSteps, sh, base);
      } else if constexpr (kForm == kBatchDf64) {
        run_steps_df64<B, W, true>(s_cs, s_cs, tm, run, sh, base);
      } else {
        if (s_cs.precision == LFM_MIXED)
          run_steps_mixed_any<B, W>(s_cs, s_cs, tm, run, kModeSteps, sh, base);
        else if (s_cs.precision == LFM_DF64)
          run_steps_df64<B, W, true>(s_cs, s_cs, tm, run, sh, base);
        else
          run_steps_f64<B, W>(s_cs, s_cs, tm, run, kModeSteps, sh, base);
      }
    }
    __syncthreads();
    if (run > 0 && tm.rank == 0 && threadIdx.x == 0) case_step[c] = base + run;
    __syncthreads();
  }
}

// Before an advance: every member case's barrier words and step counter start at zero.
__global__ void batch_prepare_kernel(const CaseDev* __restrict__ cases, int n_cases, int32_t* case_step) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_cases) {
    SyncWords* sw = cases[i].sync;
    sw->count = 0;
    sw->status = 0;
    case_step[i] = 0;
    // forms that update the FP64 field directly leave the triple-float one stale
    const int prec = cases[i].precision;
    if (prec == LFM_FP64 || (prec == LFM_MIXED && !mixed_uses_df(cases[i]))) cases[i].flags[0] = 0;
  }
}

// After an advance: each case's status, the iterations of its last step, the steps it ran
// and the iterations summed over them, gathered for one copy to the host.
__global__ void batch_collect_kernel(const CaseDev* __restrict__ cases, int n_cases,
                                     const int32_t* __restrict__ case_step, int32_t* status, int32_t* iters,
                                     int32_t* steps, int32_t* iters_sum) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n_cases) {
    status[i] = cases[i].sync->status;
    const int k = case_step[i];
    iters[i] = k > 0 ? cases[i].stats[k - 1].iters : -1;
    int sum = 0;
    for (int j = 0; j < k; ++j) sum += cases[i].stats[j].iters;
    steps[i] = k;
    iters_sum[i] = sum;
  }
}

template <int B>
void* batch_fn_w(int W, int form) {
  if (W != 6) return (void*)batch_kernel<B, 0, kBatchAny>;
  if (form == kBatchFp64) return (void*)batch_kernel<B, 6, kBatchFp64>;
  if (form == kBatchDf64) return (void*)batch_kernel<B, 6, kBatchDf64>;
  return (void*)batch_kernel<B, 6, kBatchAny>;
}

void* batch_fn(int threads, int W, int form) {
  switch (threads) {
    case 256: return batch_fn_w<256>(W, form);
    case 512: return batch_fn_w<512>(W, form);
    default: return nullptr;
  }
}

// Dynamic shared memory of a batched kernel: the stages of the bulk-staged FP32 A p, for the
// kernel that runs mixed cases (six slots).
unsigned batch_dyn_smem(int threads, int W, int form) {
  if (W != 6 || form != kBatchAny) return 0;
  switch (threads) {
    case 256: return stage_bytes_f32<256, 6>();
    case 512: return stage_bytes_f32<512, 6>();
    default: return 0;
  }
}

}  // namespace

int max_coresident_batch_ctas(int threads, int W, int form, int device) {
  void* fn = batch_fn(threads, W, form);
  if (!fn) return 0;
  int per_sm = 0, sms = 0;
  const unsigned dyn = batch_dyn_smem(threads, W, form);
  if (allow_dyn_smem(fn, dyn) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, dyn) != cudaSuccess)
    return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
  const int n = per_sm * sms;
  return n < kMaxCtas ? n : kMaxCtas;
}

cudaError_t launch_batch_prepare(const CaseDev* cases, int n_cases, int32_t* case_step, cudaStream_t s) {
  if (n_cases <= 0) return cudaSuccess;
  batch_prepare_kernel<<<(n_cases + 255) / 256, 256, 0, s>>>(cases, n_cases, case_step);
  return cudaGetLastError();
}

cudaError_t launch_batch_collect(const CaseDev* cases, int n_cases, const int32_t* case_step, int32_t* status,
                                 int32_t* iters, int32_t* steps, int32_t* iters_sum, cudaStream_t s) {
  if (n_cases <= 0) return cudaSuccess;
  batch_collect_kernel<<<(n_cases + 255) / 256, 256, 0, s>>>(cases, n_cases, case_step, status, iters, steps,
                                                              iters_sum);
  return cudaGetLastError();
}

// One batch step (or n fused steps): reset the ticket counter, then the cooperative launch.
// Written with cudaLaunchKernelEx so that it can be captured into a CUDA graph.
cudaError_t launch_batch_steps(const BatchLaunch& bl, int n_steps, cudaStream_t s) {
  void* fn = batch_fn(bl.launch.threads, bl.W, bl.form);
  if (!fn) return cudaErrorInvalidValue;
  // the opt-in above 48 KB was made when the launch shape was sized (max_coresident_batch_ctas),
  // outside any stream capture; this call finds it recorded
  const unsigned dyn = bl.launch.stage_rows ? batch_dyn_smem(bl.launch.threads, bl.W, bl.form) : 0u;
  cudaError_t e = allow_dyn_smem(fn, dyn);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(&bl.hdr->ticket, 0, sizeof(int32_t), s);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(bl.launch.ctas);
  cfg.blockDim = dim3(bl.launch.threads);
  cfg.dynamicSmemBytes = dyn;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const CaseDev* a0 = bl.cases;
  const int32_t* a1 = bl.job_case;
  const int32_t* a2 = bl.job_start;
  BatchHeader* a3 = bl.hdr;
  int32_t* a4 = bl.case_step;
  const int32_t* a5 = bl.case_cap;
  Launch a6 = bl.launch;
  int a7 = n_steps;
  void* args[] = {&a0, &a1, &a2, &a3, &a4, &a5, &a6, &a7};
  return cudaLaunchKernelExC(&cfg, fn, args);
}

#ifdef LFM_CHECKED
int check_take_batch(cudaStream_t s) {
  int site = 0;
  const int zero = 0;
  if (cudaMemcpyFromSymbolAsync(&site, g_check_site, sizeof(int), 0, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyToSymbolAsync(g_check_site, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyToSymbolAsync(g_check_inject, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return -1;
  return site;
}

void check_inject_batch(int site, cudaStream_t s) {
  cudaMemcpyToSymbolAsync(g_check_inject, &site, sizeof(int), 0, cudaMemcpyHostToDevice, s);
  cudaStreamSynchronize(s);
}
#else
int check_take_batch(cudaStream_t) { return 0; }
void check_inject_batch(int, cudaStream_t) {}
#endif

}  // namespace lfm

// Internal structures shared by the host-side C ABI (lfm_api.cu) and the kernels
// (lfm_step.cu). Nothing here is part of the public ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/lapfoam.h"

namespace lfm {

constexpr int kMaxSums = 4;          // scalars reduced per team barrier
constexpr int kMaxCtas = 8192;       // capacity of the per-CTA partial-sum table
constexpr int kStatsCap = 1024;      // per-launch statistics records
constexpr int kMaxSweeps = 5;        // mixed precision: defect-correction sweeps per step
constexpr int kMaxSlots = 32;        // largest number of internal faces per cell
constexpr int kStaticMaxCells = 1 << 16;   // allocation-free solve: largest system
constexpr int kStaticMaxFaces = 1 << 18;

// Barrier words of one team of CTAs; each field sits on its own 128-byte line.
struct alignas(128) SyncWords {
  unsigned int count;                // arrivals at the current barrier
  unsigned int pad0[31];
  unsigned int gen;                  // barrier generation (released by the last arrival)
  unsigned int pad1[31];
  double scalars[kMaxSums];          // reduced values published by the last arrival
  double pad2[16 - kMaxSums];
  int32_t status;                    // first error of the launch (0 = none)
  int32_t pad3[31];
  unsigned long long phase_ns[8];    // time per phase kind, accumulated by the team's rank 0
  unsigned long long staged;         // passes that ran with rows staged in shared memory (rank 0)
  unsigned long long pad4[7];
};

// Phase kinds of the step (indices of SyncWords::phase_ns).
enum Phase { kPhAssembly = 0, kPhInit = 1, kPhP = 2, kPhM = 3, kPhU = 4, kPhCorrect = 5, kPhases = 8 };

// Device view of one case: every pointer is device memory of the case's workspace.
struct CaseDev {
  int32_t N, F, NB;
  int32_t precision;
  double dt;
  double tol, rel_tol;
  int32_t max_iter, min_iter;

  // face-to-cell addressing, slot-major ("ELL"): each cell has W slots, slot k of cell c at
  // index k*N + c. Slots hold the cell's neighbour-side faces (ascending face id), then its
  // owned faces (ascending), then padding (other = c, face = -1, coefficient 0).
  int32_t W;
  const int32_t* slot_other; // [W*N] the other cell of the slot's face
  const int32_t* slot_face;  // [W*N] face id, -1 for padding
  const uint32_t* face_slots; // [2F] face f sits at slot face_slots[2f] (= k*N + owner) of
                              // its owner's row and at face_slots[2f+1] of its neighbour's
  const int32_t* b_start;    // [N+1] boundary faces of c: b_face[b_start[c] ..)
  const int32_t* b_face;     // [NB]  boundary faces sorted by cell, ascending id per cell
  const int32_t* bcell;      // [NB]  cell of boundary face b

  // geometry and properties
  const double* V;           // [N]
  const double* vdt;         // [N]  V/dt, recomputed whenever dt or the mesh changes
  const double* magSf;       // [F]
  const double* delta;       // [F]
  const double* DT;          // [F]
  double DT_uniform;         // the value of every DT[f] when DT_is_uniform
  int32_t DT_is_uniform;
  const double* bmagSf;      // [NB]
  const double* bdelta;      // [NB]
  const double* bDT;         // [NB]
  const double* bval;        // [NB]  fixedValue values
  const int32_t* btype;      // [NB]  LFM_FIXED_VALUE / LFM_ZERO_GRADIENT

  // general (non-orthogonal) geometry; null for orthogonal meshes. With it, delta holds the
  // implicit (nonOrthDeltaCoeffs) coefficients and the corrected laplacian adds an explicit
  // flux DT |Sf| k_f . (w_f G_P + (1 - w_f) G_N) from the Gauss gradient G of the current T.
  const double* Sf;          // [3F] internal face area vectors, owner -> neighbour (x,y,z)
  const double* fw;          // [F]  interpolation weight of the owner value
  const double* corr;        // [3F] correction vectors k_f (x,y,z)
  const double* bSf;         // [3NB] boundary face area vectors, outward (x,y,z)
  // Both are linear in T, so they are applied as operators whose weights are built from the
  // geometry (and the case's patches and DT) when those change. Component-major layout:
  // component d of cell c at d*N + c, of slot k of cell c at d*W*N + k*N + c.
  //   G_c = gD_c T_c + gH_c + sum_k gE_ck T_other(k)
  //   correction source of row c = cK_c . G_c + sum_k cL_ck . G_other(k)
  const double* gE;          // [3*W*N] (geometry only; shared with meshes that share this one)
  const double* gD;          // [3N]
  const double* gH;          // [3N]    fixedValue boundary faces
  const double* cK;          // [3N]
  const double* cL;          // [3*W*N]
  double* grad;              // [3N]    Gauss gradient of T (per assembly), component-major
  double* x_old;             // [N]  T at the start of the step (non-orthogonal correctors)
  // volumetric source S_T = Su + Sp T of Eq. (1) (fvOptions), times V; null when unset:
  // the row gets source += V Su, diag -= V Sp
  const double* vSu;         // [N]
  const double* vSp;         // [N]
  int32_t n_corr;            // extra corrector passes per step (nNonOrthogonalCorrectors)

  // assembled matrix (FP64): LDU (diag, upper) plus the per-slot copy of the off-diagonals
  double* diag;              // [N]
  double* upper;             // [F]  (lower == upper)
  double* slot_coef;         // [W*N]
  double* src;               // [N]  (FP64 steps write it only for matrix read-back)
  double* rD;                // [N]  1/diag

  // FP64 solver vectors; x is the field T (updated in place)
  double* x;
  double* r;
  double* w;
  double* p;
  double* q;

  // mixed precision: FP32 matrix copy and inner-solve vectors
  float* diag32;
  float* slot_coef32;        // [W*N]
  float* rD32;
  float* dx32;
  float* r32;
  float* w32;
  float* p32;
  float* q32;

  // df64 form (lfm_solve_df.cuh): the diagonal and its reciprocal, V/dt and the per-slot
  // face conductances as double-float pairs (hi, lo), all scaled by df_scale (a power of
  // two), and the field as a triple-float; r, w, p, q and x_old are used as float2 arrays of
  // the same size
  float2* x2;                // [N]   field: leading and middle parts of a triple-float
  float* xlo;                // [N]   field: trailing part
  float* xolo;               // [N]   trailing part of x_old (x_old holds the other two)
  float2* e2;                // [N]   the current solve's correction to the field
  int32_t* flags;            // [2]   flags[0] != 0: the triple-float field (x2, xlo) is current and
                             //       x holds its rounding; 0: x was written otherwise (split it).
                             //       flags[1] != 0: the mixed form's last launch ended with the
                             //       next step's rows and inner-solve seed in place (seed_sums);
                             //       cleared by every host change to the case
  double* seed_sums;         // [3]   their team totals: normFactor sum, sum|r|, rho
  float2* diag2;             // [N]
  float2* rD2;               // [N]
  const float2* vdt2;        // [N]   V/dt * df_scale
  const float2* g2;          // [W*N] DT |Sf| deltaCoeff * df_scale at both slots of each face
  double df_scale;
  // df64 form on general geometry: the operator weights gE (gradient) and cK, cL (correction,
  // times df_scale) as pairs, the closure weight gZ = gD + sum_k gE_k + sum_fixedValue bSf / V
  // (formed in FP64; zero for a closed cell up to rounding) of the gradient's difference form,
  // and the gradient itself (component-major as the FP64 arrays)
  const float2* gE2;         // [3*W*N]
  const float2* cK2;         // [3N]
  const float2* cL2;         // [3*W*N]
  const float2* gZ;          // [3N]   (pairs of the FP64 closure weight)
  float2* grad2;             // [3N]

  // team state
  SyncWords* sync;
  double* partials;          // [kMaxCtas * kMaxSums]
  lfm_step_stats* stats;     // [kStatsCap]
};

struct Launch {
  int ctas;
  int threads;
  uint64_t timeout_ns;
  int skip_cta;              // test hook: CTA that leaves before its first arrival (-1: none)
  int stage_rows;            // 0: passes load their matrix rows into registers (test switch)
  int skip_copy_cta;         // test hook: CTA that issues no copy for its first staged tile (-1: none)
};

enum Mode { kModeSteps = 0, kModeAssembleOnly = 1 };

// Batched form: job table header in device memory (rewritten before each advance).
struct BatchHeader {
  int32_t n_jobs;
  int32_t n_tickets;
  int32_t ticket;            // next ticket; reset to 0 before every launch
  int32_t pad;
};

struct BatchLaunch {
  const CaseDev* cases;      // [n_cases] descriptors of the member cases
  const int32_t* job_case;   // [n_jobs] case of job j
  const int32_t* job_start;  // [n_jobs + 1] first ticket of job j
  BatchHeader* hdr;
  int32_t* case_step;        // [n_cases] steps done in the current advance
  const int32_t* case_cap;   // [n_cases] at most this many steps of the current advance
  Launch launch;
  int W;
  int form;  // kBatchAny, or the one precision every member runs (kernel compiled for it)
};

// Kernel variants of the batched step: any member precision, or FP64 / df64 members only
// (the single-form kernels carry only their form's passes: less code around the iteration
// loops; slot width 6 only).
enum BatchForm { kBatchAny = 0, kBatchFp64 = 1, kBatchDf64 = 2 };

// Kernel launchers (lfm_step.cu). Return a cudaError_t.
cudaError_t launch_steps(const CaseDev& cs, const Launch& L, int n_steps, int mode,
                         cudaStream_t stream);
// Largest co-resident CTA count for the step kernel at `threads` per CTA.
// Opts a kernel into more than 48 KB of dynamic shared memory (once per kernel and device).
cudaError_t allow_dyn_smem(void* fn, unsigned bytes);
int max_coresident_ctas(int precision, int threads, int W, int device);
cudaError_t launch_boundary_values(const CaseDev& cs, double* Tb, cudaStream_t stream);
// Gauss linear gradient of the current T: cells into cs.grad, and (bgrad non-null) the
// corrected boundary values [3NB] (x,y,z per face).
cudaError_t launch_grad(const CaseDev& cs, double* bgrad, cudaStream_t stream);
// Operator weights of the general-geometry path: gE (geometry only) when `with_E`, and the
// case's gD, gH, cK, cL (patches, boundary values, DT).
cudaError_t launch_geom_ops(const CaseDev& cs, bool with_E, cudaStream_t stream);
// Face diffusivities from a cell field: DTf = w (DT_P - DT_N) + DT_N, DTb = DT of the cell.
cudaError_t launch_dt_cells(const CaseDev& cs, const double* DTc, const double* w, double* DTf, double* DTb,
                            cudaStream_t stream);
// out[c] = V[c] * a[c] (a null: out = 0).
cudaError_t launch_times_volume(const CaseDev& cs, const double* a, double* out, cudaStream_t stream);
// Set-up of the face coefficients: -DT |Sf| deltaCoeff at both slots of every face in the
// FP64 slot array and, when present, the FP32 one.
cudaError_t launch_coef_setup(const CaseDev& cs, cudaStream_t stream);
// Whether the mixed form of this case runs its outer passes in df64 (orthogonal mesh, df64
// block present, scale an FP32 power of two).
bool mixed_runs_df(const CaseDev& cs);
// df64 form set-up: the per-slot conductances g2 and V/dt (vdt2), both times cs.df_scale,
// and on general geometry the operator weights gE2, cK2, cL2 and gZ (see CaseDev).
cudaError_t launch_df_setup(const CaseDev& cs, cudaStream_t stream);

// Face-to-cell addressing of a general mesh built on the device (lfm_addr.cu): owner,
// neighbour, bface_cell are device arrays; W the largest internal-face count of a cell.
cudaError_t build_addressing(int32_t N, int32_t F, int32_t NB, int32_t W, const int32_t* owner,
                             const int32_t* neighbour, const int32_t* bface_cell, int32_t* slot_other,
                             int32_t* slot_face, uint32_t* face_slots, int32_t* b_start, int32_t* b_face,
                             cudaStream_t stream);

// Box meshes built from closed forms (lfm_box.cu).
int box_slot_width(long long nx, long long ny, long long nz);
cudaError_t launch_box(long long nx, long long ny, long long nz, int W, const double* xs, const double* ys,
                       const double* zs, const CaseDev& cs, cudaStream_t stream);
void box_layout_host(long long nx, long long ny, long long nz, int W, const double* xs, const double* ys,
                     const double* zs, int32_t* slot_other, int32_t* slot_face, uint32_t* face_slots,
                     double* V, double* magSf,
                     double* delta, int32_t* b_start, int32_t* b_face, int32_t* bcell, double* bmagSf,
                     double* bdelta);

// Batched launchers (lfm_batch.cu).
int max_coresident_batch_ctas(int threads, int W, int form, int device);
cudaError_t launch_batch_prepare(const CaseDev* cases, int n_cases, int32_t* case_step, cudaStream_t s);
// After an advance, per case: status, iterations of its last step (-1: none), steps run and
// iterations summed over them.
cudaError_t launch_batch_collect(const CaseDev* cases, int n_cases, const int32_t* case_step, int32_t* status,
                                 int32_t* iters, int32_t* steps, int32_t* iters_sum, cudaStream_t s);
cudaError_t launch_batch_steps(const BatchLaunch& bl, int n_steps, cudaStream_t s);
cudaError_t launch_fill(double* a, size_t n, double v, cudaStream_t stream);
cudaError_t launch_vdt(const double* V, double dt, double* vdt, int n, cudaStream_t stream);

// ---- one case decomposed into parts (lfm_decomp.cu) ------------------------------------
// Plan of part s of a decomposition into P contiguous label ranges: its first label and
// owned count, its ghost labels (sorted), and what it sends: for each of its interface
// cells (local id, ascending) every (part, ghost slot) that mirrors it.
struct DdPlanPart {
  int32_t first = 0, n_owned = 0;
  std::vector<int32_t> ghost;
  std::vector<int32_t> send_src, send_part, send_slot;
};
int32_t dd_first_label(int32_t N, int32_t P, int32_t s);
int32_t dd_part_of(int32_t N, int32_t P, int32_t label);
void dd_plan_from_faces(int32_t N, int32_t F, const int32_t* owner, const int32_t* neighbour, int32_t P,
                        int32_t s, DdPlanPart& out);
void dd_plan_from_slots(int32_t N, int32_t W, const int32_t* slot_other, int32_t P, int32_t s, DdPlanPart& out);

// Device view of one part: its rows are the global rows [first, first + N) (coefficients and
// boundary data read from the case's arrays); its columns are local (owned < N <= ghost);
// its vectors are its own (T and p with N + G entries, the ghosts after the owned cells).
struct DdPart {
  int32_t N, G, first, n_send, ctas;
  const int32_t* slot_local;  // [W*N]
  const int32_t* send_src;    // [n_send] local owned id, ascending
  const int32_t* send_part;   // [n_send] receiving part
  const int32_t* send_slot;   // [n_send] ghost slot in the receiving part
  double* x;                  // [N + G]
  double* p;                  // [N + G]
  double* r;                  // [N]
  double* w;
  double* q;
  double* diag;
  double* rD;
};
int dd_max_ctas(int threads, int W, int device);
cudaError_t launch_dd_steps(const CaseDev& cs, const DdPart* parts, const int32_t* cta_part, const int32_t* cta_rank,
                            const Launch& L, int n_steps, cudaStream_t stream);

// Records the reason for a failed context-free call (the text lfm_last_error(NULL) returns
// on this thread); defined with the thread-local error text in lfm_api.cu. Returns code.
int set_last_error(int code, const char* fmt, ...);

// Index checks of the checked build (lfm_device.cuh), per kernel translation unit: take
// returns the first failing check site recorded on the current device since the last take
// (0: none) and clears it and the injection hook; inject makes `site` report as failing
// (one-shot: the next take clears it). Without LFM_CHECKED, take returns 0 and inject does
// nothing.
#ifdef LFM_CHECKED
constexpr bool kCheckedBuild = true;
#else
constexpr bool kCheckedBuild = false;
#endif
int check_take_step(cudaStream_t s);
int check_take_batch(cudaStream_t s);
void check_inject_step(int site, cudaStream_t s);
void check_inject_batch(int site, cudaStream_t s);

}  // namespace lfm

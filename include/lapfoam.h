/*
 * lapfoam.h -- C ABI of liblapfoam.so: one implicit-Euler time step of laplacianFoam
 * (arXiv 2507.18268) on an NVIDIA GB300 (sm_103a).
 *
 * What a step computes (paper, section "The laplacianFoam application", Eq. (1) and the
 * listing "laplacianFoam application"): the matrix of fvm::ddt(T) - fvm::laplacian(DT, T)
 * is assembled in OpenFOAM's LDU face-addressed form (section "OpenFOAM": owner and
 * neighbour per internal face, faces in upper-triangular order) and solved by the
 * conjugate-gradient method with the diagonal preconditioner (section "Evaluation"),
 * stopping on OpenFOAM's normFactor-scaled L1 residual.
 *
 * Conventions shared by every call:
 *   - Every call returns an int status (LFM_OK = 0 or a negative LFM_E* code); no C++
 *     exception crosses this boundary. lfm_last_error() gives a one-line reason.
 *   - Host arrays passed in are read during the call only (deep copy); the caller keeps
 *     ownership. Output arrays are caller-allocated host memory unless said otherwise.
 *   - A context holds one case on one device and issues all its work on one CUDA stream
 *     (the one passed to lfm_create; NULL = the legacy default stream). A context is not
 *     thread-safe; distinct contexts may be used from distinct threads.
 *   - Device memory is either a caller-bound workspace (lfm_bind_workspace, never freed by
 *     the library) or allocated by the library at upload time and freed by lfm_destroy.
 *   - Non-convergence within max_iter is reported in the step statistics, not as an error
 *     (as OpenFOAM does). A singular search direction (|p.Ap| / normFactor < 1e-300) stops
 *     the step and returns LFM_ESINGULAR; a non-finite residual returns LFM_ENONFINITE.
 *   - Calls made out of order (advance before upload, ...) return LFM_ESTATE.
 */
#ifndef LAPFOAM_H
#define LAPFOAM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  LFM_OK = 0,
  LFM_EINVAL = -1,     /* bad argument or mesh (index out of range, owner >= neighbour, V <= 0, NaN) */
  LFM_ENOMEM = -2,     /* workspace too small / device allocation failed / over budget */
  LFM_ECUDA = -3,      /* a CUDA runtime call failed */
  LFM_ESINGULAR = -4,  /* PCG met a singular search direction */
  LFM_ENONFINITE = -5, /* residual became NaN/Inf */
  LFM_ETIMEOUT = -6,   /* a device-side barrier wait gave up (kernel returned; context usable) */
  LFM_ESTATE = -7      /* call out of order */
};

enum { LFM_FIXED_VALUE = 0, LFM_ZERO_GRADIENT = 1 };
/* Arithmetic of the step (lfm_solver_opts.precision):
 *   LFM_FP64   IEEE FP64 throughout; the assembled system is bitwise the CPU reference's.
 *   LFM_MIXED  FP32 inner CG inside FP64-class defect correction (results ~1e-6 relative):
 *              the outer passes (true residual, correction) use the LFM_DF64 machinery on
 *              orthogonal meshes and FP64 on general ones. Within one advance, each step's
 *              verification pass also assembles the next step (no sources or correctors);
 *              results equal those of one-step advances bit for bit.
 *   LFM_DF64   every per-cell operation in double-float (pairs of FP32 numbers, 48-bit
 *              significand) on the FP32 pipe, per-CTA scalars in FP64: results agree with
 *              FP64 to rounding (~1e-13 relative), at FP32-pipe speed; any mesh (general
 *              geometry included), DT, sources and corrector passes. */
enum { LFM_FP64 = 0, LFM_MIXED = 1, LFM_DF64 = 2 };

typedef struct lfm_ctx lfm_ctx;

/*
 * LDU mesh (section "OpenFOAM" of the paper: owner/neighbour face addressing).
 *   owner[f] < neighbour[f] for every internal face f, faces sorted by (owner, neighbour)
 *   (upper-triangular order). V[c] > 0 cell volumes, magSf[f] > 0 face areas,
 *   deltaCoeffs[f] > 0 the inverse owner-to-neighbour centre distance.
 *   Boundary faces are grouped in patches: patch p covers boundary faces
 *   [patch_start[p], patch_start[p] + patch_size[p]) which must tile [0, n_bfaces) in order.
 *   bface_cell[b] is the cell of boundary face b, bmagSf its area, bdeltaCoeffs the inverse
 *   distance from the cell centre to the face centre.
 * All arrays are host memory, int32 indices, float64 values.
 */
typedef struct {
  int32_t n_cells, n_faces;
  const int32_t *owner, *neighbour;
  const double *V, *magSf, *deltaCoeffs;
  int32_t n_patches;
  const int32_t *patch_start, *patch_size;
  int32_t n_bfaces;
  const int32_t *bface_cell;
  const double *bmagSf, *bdeltaCoeffs;
} lfm_mesh;

/*
 * Geometry of a general (non-orthogonal) hexahedral or polyhedral mesh, for the corrected
 * laplacian and the Gauss linear gradient (section "Code Porting" of the paper: the
 * interpolation weights, dotInterpolate, the two gradf cycles, the division by the cell
 * volume and correctBoundaryConditions).
 *   Sf[3*n_faces]        internal face area vectors (x, y, z per face), owner -> neighbour;
 *                        |Sf| must equal the mesh's magSf (relative 1e-9);
 *   weights[n_faces]     linear-interpolation weight of the owner value, in [0, 1]: the
 *                        face value is w (T_P - T_N) + T_N;
 *   corr_vec[3*n_faces]  non-orthogonal correction vectors k = Sf/|Sf| - d * deltaCoeffs
 *                        (d = C_N - C_P);
 *   bSf[3*n_bfaces]      boundary face area vectors, pointing out of the domain.
 * With it the mesh's deltaCoeffs are the implicit (non-orthogonal) coefficients
 * 1 / max(n.d, 0.05 |d|) and bdeltaCoeffs the inverse patch-normal distances. The laplacian
 * of every assembly then adds the explicit flux DT |Sf| k . (w (G_P - G_N) + G_N), G the
 * Gauss gradient of the current T, to the source (boundary faces carry no correction).
 * Host memory, float64; copied at upload.
 */
typedef struct {
  const double *Sf, *weights, *corr_vec, *bSf;
} lfm_geometry;

/* PCG controls. tol: stop when sum|r| / normFactor < tol; rel_tol > 0 also stops when the
 * residual falls below rel_tol times the step's initial residual; max_iter caps and
 * min_iter forces iterations (OpenFOAM defaults: 1000, 0). precision: LFM_FP64,
 * LFM_MIXED (FP32 matrix and vectors, FP64-accurate dots / normFactor / convergence test /
 * true residual, field updated by defect correction) or LFM_DF64 (see above). */
typedef struct {
  double tol, rel_tol;
  int32_t max_iter, min_iter, precision;
} lfm_solver_opts;

/* Per-step solver record. iters: PCG iterations (LFM_MIXED: inner FP32 iterations summed
 * over the refinement sweeps); sweeps: LFM_MIXED refinement sweeps (LFM_FP64: 1, or 0 when
 * the step needed no iteration); init_res / final_res: normFactor-scaled L1 residuals
 * (LFM_MIXED: of the FP64 true residual b - A T). With non-orthogonal correctors (see
 * lfm_set_nonorth_correctors) a step runs several assemble-and-solve passes: iters and
 * sweeps are summed over them, init_res and norm_factor are the first pass's, final_res
 * and converged the last pass's. */
typedef struct {
  int32_t iters, converged, sweeps, status;
  double init_res, final_res, norm_factor;
} lfm_step_stats;

/* Library version string. */
const char *lfm_version(void);

/* ---- host-only helpers (no device is touched) ------------------------------------- */

/* Validates a mesh: index ranges, owner < neighbour, upper-triangular order, positive
 * finite geometry, patches tiling the boundary faces. Returns LFM_OK or LFM_EINVAL with the
 * reason in msg (msg may be NULL). */
int lfm_mesh_check(const lfm_mesh *mesh, char *msg, size_t msg_len);

/* Face-to-cell addressing of the paper's section "Code Porting" (lists of lists built once
 * per mesh): for cell c, its owner-side faces are [own_start[c], own_start[c+1]) (faces are
 * sorted by owner), and its neighbour-side faces are losort[lo_start[c] .. lo_start[c+1])
 * in ascending face order. own_start, lo_start: n_cells+1 entries; losort: n_faces.
 * Counting sort, O(n_cells + n_faces). Input must satisfy lfm_mesh_check. */
int lfm_face_addressing(int32_t n_cells, int32_t n_faces, const int32_t *owner,
                        const int32_t *neighbour, int32_t *own_start, int32_t *losort,
                        int32_t *lo_start);

/* Box meshes (rectilinear hexahedra, natural numbering c = i + nx (j + ny k), vertex
 * coordinates xs[nx+1], ys[ny+1], zs[nz+1] strictly increasing; patches x0, x1, y0, y1,
 * z0, z1 with x-patch faces ordered by (k, j), y-patch by (k, i), z-patch by (j, i)).
 * Counts of such a mesh: cells, internal faces, boundary faces, slots per cell. */
int lfm_box_counts(int32_t nx, int32_t ny, int32_t nz, int32_t *n_cells, int32_t *n_faces,
                   int32_t *n_bfaces, int32_t *slot_width);

/* Host replica of the device box builder (same per-cell routine): fills the slot-major
 * face-to-cell arrays (slot_other, slot_face [W*N]: slot k of cell c at k*N + c), the
 * per-face slot positions (face_slots [2F]: face f sits at slot face_slots[2f] of its
 * owner's row and at face_slots[2f+1] of its neighbour's row), V [N], magSf,
 * deltaCoeffs [F], the cell-side boundary lists (b_start [N+1], b_face [NB]) and
 * bface_cell, bmagSf, bdeltaCoeffs [NB]. For validation of the closed forms; no device is
 * touched. Boxes with W*N >= 2^32 are rejected (LFM_EINVAL). */
int lfm_box_layout(int32_t nx, int32_t ny, int32_t nz, const double *xs, const double *ys,
                   const double *zs, int32_t *slot_other, int32_t *slot_face, uint32_t *face_slots,
                   double *V, double *magSf, double *deltaCoeffs, int32_t *b_start, int32_t *b_face,
                   int32_t *bface_cell, double *bmagSf, double *bdeltaCoeffs);

/* ---- single-case context ----------------------------------------------------------- */

/* Device bytes lfm_upload_mesh needs for this mesh: precision LFM_FP64, LFM_MIXED or
 * LFM_DF64 for a workspace serving that precision only (an LFM_DF64 workspace also serves
 * LFM_FP64), any other value (e.g. -1) for one serving all three.
 * A library-owned workspace (no lfm_bind_workspace) always serves all three. */
size_t lfm_workspace_bytes(const lfm_mesh *mesh, int32_t precision);

/* Creates a context on CUDA device `device`, issuing work on `cuda_stream` (a
 * cudaStream_t; NULL = legacy default stream). */
int lfm_create(lfm_ctx **out, int device, void *cuda_stream);

/* Binds caller-owned device memory that upload carves all device arrays from: at least
 * lfm_workspace_bytes(mesh, precision) bytes, 256-byte aligned; `precision` (LFM_FP64,
 * LFM_MIXED, LFM_DF64, or -1 for all) selects which solver buffers it holds, and lfm_set_solver
 * refuses a precision it does not hold (LFM_ENOMEM). Must precede lfm_upload_mesh; the
 * library never frees it. */
int lfm_bind_workspace(lfm_ctx *ctx, void *dev_ptr, size_t bytes, int32_t precision);

/* Device bytes lfm_upload_mesh_geometry needs (the general-geometry arrays, and per case
 * the gradient [3N] and correction flux [F]); precision as for lfm_workspace_bytes. */
size_t lfm_workspace_bytes_geometry(const lfm_mesh *mesh, int32_t precision);

/* Validates and uploads the mesh (deep copy), builds the face-to-cell addressing and the
 * cell-side boundary-face lists on the device (section "Code Porting": the lists of lists,
 * by binary search over the owner-sorted faces, a counting sort by neighbour and by boundary
 * cell -- atomic counts, scan, placement, per-cell sort -- and the slot-major rows). Resets DT to 0, every patch to zeroGradient, dt to 1,
 * the solver to {1e-6, 0, 1000, 0, LFM_FP64} and T to 0. LFM_EINVAL also when a cell has
 * more than 32 internal faces or (largest internal faces of a cell) x n_cells >= 2^32. */
int lfm_upload_mesh(lfm_ctx *ctx, const lfm_mesh *mesh);

/* As lfm_upload_mesh, for a general (non-orthogonal) mesh: also uploads `geometry` and
 * switches the laplacian to its corrected form. LFM_EINVAL when the geometry is
 * inconsistent with the mesh (see lfm_geometry). */
int lfm_upload_mesh_geometry(lfm_ctx *ctx, const lfm_mesh *mesh, const lfm_geometry *geometry);

/* Number of extra non-orthogonal corrector passes per time step (OpenFOAM's
 * nNonOrthogonalCorrectors; laplacianFoam's listing loops over them): every step assembles
 * and solves 1 + n_corr times, each pass with the explicit correction from the latest T and
 * the ddt source from T at the start of the step. 0 after upload; 0..64. Allowed on any
 * mesh (on an orthogonal one the correction is zero and the extra passes re-solve). */
int lfm_set_nonorth_correctors(lfm_ctx *ctx, int32_t n_corr);

/* Gauss linear gradient of the current T (section "Code Porting": face values by linear
 * interpolation or the boundary values, the Gauss sum over internal and boundary faces,
 * division by V): grad[3*n_cells] (x, y, z per cell) to host memory; bgrad[3*n_bfaces]
 * (may be NULL) receives the boundary values after correctBoundaryConditions (the cell's
 * gradient with its normal component replaced by the patch snGrad). LFM_ESTATE without
 * general geometry or with an advance pending. */
int lfm_grad(lfm_ctx *ctx, double *grad, double *bgrad);

/* Builds a box mesh (see lfm_box_counts) directly on the device -- the same arrays as
 * uploading the equivalent LDU mesh with lfm_upload_mesh, from closed forms, one thread
 * per cell -- and resets properties and controls like lfm_upload_mesh. */
int lfm_upload_box(lfm_ctx *ctx, int32_t nx, int32_t ny, int32_t nz, const double *xs,
                   const double *ys, const double *zs);

/* Workspace bytes for lfm_upload_box (precision as in lfm_workspace_bytes). */
size_t lfm_workspace_bytes_box(int32_t nx, int32_t ny, int32_t nz, int32_t precision);

/* Mesh sharing (for many cases on one mesh, e.g. a server): the context uses the mesh
 * arrays (face-to-cell slots, boundary lists, geometry) uploaded by `src` instead of its
 * own copy, and owns only its per-case arrays (properties, boundary values, matrix,
 * field, solver vectors). `src` must stay alive (lfm_destroy refuses it while sharers
 * exist). Resets properties and controls like lfm_upload_mesh. */
int lfm_upload_mesh_shared(lfm_ctx *ctx, lfm_ctx *src);

/* Workspace bytes of a context sharing src's mesh (precision as in lfm_workspace_bytes). */
size_t lfm_workspace_bytes_shared(const lfm_ctx *src, int32_t precision);

/* Sets every cell of T to `value` on the device. */
int lfm_fill_field(lfm_ctx *ctx, double value);

/* Diffusivity DT per internal face (DT_faces[n_faces]) and per boundary face
 * (DT_bfaces[n_bfaces]); a NULL array takes the value `uniform`. Values must be finite
 * and >= 0. */
int lfm_set_diffusivity(lfm_ctx *ctx, double uniform, const double *DT_faces,
                        const double *DT_bfaces);

/* Diffusivity as a cell field DT_cells[n_cells] >= 0 (a volScalarField DT in Eq. (1)): each
 * internal face takes the linear interpolate w (DT_P - DT_N) + DT_N (the dotInterpolate form
 * of section "Code Porting"), each boundary face the value of its cell. weights[n_faces] in
 * [0, 1] are the owner weights (NULL: those of the uploaded general geometry; LFM_EINVAL when
 * there is none). Computed on the device; replaces any earlier diffusivity. */
int lfm_set_diffusivity_cells(lfm_ctx *ctx, const double *DT_cells, const double *weights);

/* Volumetric source S_T = Su + Sp T of Eq. (1) per unit volume (OpenFOAM's fvOptions, e.g. a
 * semi-implicit source), on the right-hand side: every assembly adds V Su to the source and
 * -V Sp to the diagonal (Sp <= 0 keeps the matrix diagonally dominant). Su, Sp: host arrays
 * [n_cells] or NULL (0); both NULL removes the source. */
int lfm_set_source(lfm_ctx *ctx, const double *Su, const double *Sp);

/* Patch type (LFM_FIXED_VALUE / LFM_ZERO_GRADIENT) and, for fixedValue, the boundary
 * values: values[patch_size[patch]] or, when values is NULL, `uniform` on every face. The
 * boundary conditions of T in Eq. (1) (section "The laplacianFoam application": T is read
 * with its patch types): a fixedValue face adds its conductance DT|Sb|/|C_b - C_P| to the
 * diagonal and that times the value to the source; a zeroGradient face adds nothing. The
 * values are deep-copied; LFM_EINVAL for a patch index or type out of range or a
 * non-finite value. */
int lfm_set_patch(lfm_ctx *ctx, int32_t patch, int32_t type, const double *values,
                  double uniform);

/* Time step deltaT of the implicit Euler ddt term of Eq. (1) (fvm::ddt(T) in the listing
 * "laplacianFoam application": V/deltaT on the diagonal, V/deltaT T_old in the source).
 * LFM_EINVAL unless finite and > 0; V/deltaT is recomputed on the device. */
int lfm_set_time_step(lfm_ctx *ctx, double dt);

/* Solver controls (tol >= 0, rel_tol >= 0, max_iter >= 1, 0 <= min_iter <= max_iter). */
int lfm_set_solver(lfm_ctx *ctx, const lfm_solver_opts *opts);

/* Field T[n_cells] from host memory (stream-ordered copy; synchronises before return). */
int lfm_set_field(lfm_ctx *ctx, const double *T);

/* Field T from device memory of the same device (T_dev[n_cells], stream-ordered). */
int lfm_set_field_device(lfm_ctx *ctx, const double *T_dev);

/* Runs n_steps implicit steps on the device: per step assemble, initial residual and
 * normFactor, PCG iterations, all inside device-side control flow; T_old <- T each step.
 * One step is one pass of the time loop in the listing "laplacianFoam application":
 * assemble TEqn = fvm::ddt(T) - fvm::laplacian(DT, T) (Eq. (1)) and solve it with the
 * diagonal-preconditioned CG named in section "Evaluation" (stopping on the normFactor-
 * scaled L1 residual). Synchronises before return; out (host, n_steps records, may be
 * NULL) receives the per-step statistics. Non-convergence is reported in the records, not
 * as an error; LFM_ESTATE before an upload, LFM_ETIMEOUT / LFM_ENONFINITE / LFM_ESINGULAR
 * from the device (the context stays usable). */
int lfm_advance(lfm_ctx *ctx, int32_t n_steps, lfm_step_stats *out);

/* Enqueues n_steps like lfm_advance without waiting (statistics stay on the device until
 * lfm_finish). At most one pending advance per context. */
int lfm_advance_async(lfm_ctx *ctx, int32_t n_steps);

/* 1 if the pending advance is still running, LFM_OK if done (or none pending). */
int lfm_query(lfm_ctx *ctx);

/* Waits for the pending advance, copies up to n records of statistics to out (may be
 * NULL) and returns its status. */
int lfm_finish(lfm_ctx *ctx, lfm_step_stats *out, int32_t n);

/* Reads T[n_cells] to host memory and, when T_boundary is not NULL, the boundary-face
 * values T_boundary[n_bfaces] (fixedValue: the set value; zeroGradient: the face cell's T),
 * both computed on the device: the field the laplacianFoam listing writes at the end of a
 * time step, with its boundary values as the patch types define them (section "Code
 * Porting": the boundary evaluation of a field). T_out is a caller-owned host buffer;
 * synchronises before return; LFM_ESTATE before an upload. */
int lfm_get_field(lfm_ctx *ctx, double *T_out, double *T_boundary);

/* Device pointer of the context's T[n_cells] (float64), valid until lfm_destroy, for reading
 * (it holds the field after every advance). Write the field with lfm_set_field,
 * lfm_set_field_device or lfm_fill_field: the LFM_DF64 and LFM_MIXED forms carry the field
 * between advances at higher precision (a triple-float) and re-read this array only after
 * one of those calls. */
int lfm_field_device_ptr(lfm_ctx *ctx, double **T_dev);

/* Reads the assembled matrix of the current T (diag[n_cells], upper[n_faces],
 * source[n_cells]) to host memory, running only the assembly. Diagnostic / test use. */
int lfm_get_matrix(lfm_ctx *ctx, double *diag, double *upper, double *source);

/* Reads back the face-to-cell addressing built at upload (diagnostic / test use): the
 * slot-major rows slot_other, slot_face [W*N] (W = lfm_box_counts' slot width for boxes, else
 * the largest number of internal faces of a cell), face_slots [2*n_faces], b_start
 * [n_cells+1], b_face [n_bfaces]; any pointer may be NULL. */
int lfm_get_addressing(lfm_ctx *ctx, int32_t *slot_other, int32_t *slot_face, uint32_t *face_slots,
                       int32_t *b_start, int32_t *b_face);

/* Device time of the last advance by phase kind, in milliseconds (ms[8]): 0 assembly pass
 * over faces (coefficients, sum of T), 1 assembly pass over rows together with the initial
 * residual / normFactor (mixed: also the later FP64 true residuals), 2 search-direction update,
 * 3 matrix-vector product and p.Ap, 4 solution/residual update and dots, 5 (mixed) FP64
 * correction, 6-7 unused. Measured by one CTA between barrier exits, so each phase
 * includes its barrier wait; the sum is the kernel's wall time. */
int lfm_get_phase_times(lfm_ctx *ctx, double *ms);

/* Launch configuration chosen by the tuner for this context: CTAs and threads per CTA. */
int lfm_get_launch(lfm_ctx *ctx, int32_t *ctas, int32_t *threads);

/* Overrides the launch configuration (ctas <= 0 or threads <= 0 restores the tuned one).
 * ctas is clamped to what can be co-resident. */
int lfm_set_launch(lfm_ctx *ctx, int32_t ctas, int32_t threads);

/* Sets the device-side barrier wait limit in nanoseconds (default 2e9). When one wait
 * runs out the kernel stops and the call returns LFM_ETIMEOUT; the context stays usable. */
int lfm_set_barrier_timeout(lfm_ctx *ctx, uint64_t ns);

/* Test hook: when cta >= 0, the next advance makes CTA `cta` leave the kernel before its
 * first barrier arrival, so the other CTAs' waits run out and the advance returns
 * LFM_ETIMEOUT (no fault, no hang: every wait is bounded). One-shot; needs >= 2 CTAs. */
int lfm_debug_skip_arrival(lfm_ctx *ctx, int32_t cta);

/* Test hook: when cta >= 0, the next advance makes CTA `cta` issue no copy for the first tile
 * of its first shared-memory-staged pass (see lfm_debug_stage_rows), so that its wait for
 * those bytes runs out and the advance returns LFM_ETIMEOUT (no fault, no hang: every wait is
 * bounded). One-shot; no effect when the launch stages no rows. */
int lfm_debug_skip_stage_copy(lfm_ctx *ctx, int32_t cta);

/* Test evidence: the number of passes of the last advance (lfm_advance / lfm_advance_async
 * and its finish) that ran with their matrix rows staged in shared memory, counted once per
 * pass on the team's first CTA; 0 when the register form ran throughout. */
int lfm_debug_staged_passes(lfm_ctx *ctx, int64_t *n);

/* Test switch: on != 0 (the default) lets the passes that can stream their matrix rows into
 * shared memory with bulk copies do so (the FP32 A p of the mixed form on orthogonal meshes,
 * in single-case launches, on meshes of six slots per cell with N a multiple of 4); 0 makes
 * them load the rows into registers. Both give the same results bit for bit; the switch exists to test
 * that. */
int lfm_debug_stage_rows(lfm_ctx *ctx, int32_t on);

/* 1 when this library is the checked build (compiled with LFM_CHECKED, liblapfoam_checked.so),
 * else 0. In the checked build every kernel tests each index it reads from the mesh's
 * addressing before using it as an address: a slot's neighbour cell (< n_cells), a face's
 * slot positions and a slot's face, a cell's boundary faces and a boundary face's cell. A
 * bad index is replaced by an in-range one and recorded; the advance (or batch finish) that
 * follows returns LFM_EINVAL naming the check site (1 slot cell, 2 face/slot, 3 boundary,
 * 4 slot cell in the df64 passes). Nothing is read or written out of bounds and nothing
 * traps, so the context stays usable. This stands in for a memory checker: the build's
 * results must equal the normal build's bit for bit. */
int lfm_checked_build(void);

/* Test hook of the checked build: makes check site `site` (1..4) report as failing, with no
 * bad index, wherever the kernels evaluate it until the next advance (or batch finish)
 * collects the checks; that call then returns LFM_EINVAL. One-shot: the collection clears
 * it. LFM_ESTATE in the normal build; LFM_EINVAL for another site number. */
int lfm_debug_check_inject(lfm_ctx *ctx, int32_t site);

/* Allocation-free solve, for callers that cannot allocate device memory (a plug-in inside a
 * host code whose memory manager owns every device buffer, a real-time loop that must not
 * call an allocator once running). The paper has no counterpart to this call.
 * Solves A x = source with the same diagonal-preconditioned CG and normFactor residual as
 * lfm_advance, FP64 only (opts->precision must be LFM_FP64), where A is given in LDU form
 * in device memory the caller owns: owner/neighbour[n_faces] (owner < neighbour, sorted by
 * owner), diag[n_cells], upper[n_faces] (lower == upper), source[n_cells]; x[n_cells]
 * (device) holds the initial guess and receives the solution. x must not overlap any input
 * array (LFM_EINVAL). stats (host, may be NULL) receives the solve record. Runs on
 * cuda_stream; every call synchronises that stream before it returns (it reads the record
 * back), so the result is in x on return.
 * Limits: n_cells <= 65536 and n_faces <= 262144, else LFM_EINVAL before any device work;
 * at most 32 internal faces per cell (as lfm_upload_mesh). A face out of range, faces not
 * sorted by owner or a cell above the face limit are reported as LFM_EINVAL by the kernel
 * before it uses any of those indices as an address; x is then left unchanged. Every
 * non-OK return sets the text of lfm_last_error(NULL) on the calling thread.
 * Working memory: one fixed device array of about 4.8 MB inside the library, present on
 * every GPU that loads it until the process exits; no call allocates, frees or calls an
 * allocating library routine. All calls share that array (each call re-initialises what it
 * needs), so calls whose kernels overlap on one GPU race: order them on one stream. The
 * first call on a device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current. Because every call synchronises its stream, no call can be part of a
 * stream capture: on a stream that is being captured the call returns LFM_ESTATE before any
 * device work (and leaves the capture intact). */
int lfm_pcg_solve_static(int32_t n_cells, int32_t n_faces, const int32_t *owner,
                         const int32_t *neighbour, const double *diag, const double *upper,
                         const double *source, double *x, const lfm_solver_opts *opts,
                         lfm_step_stats *stats, void *cuda_stream);

/* ---- one case decomposed into parts ----------------------------------------------------
 * The data flow of the paper's multi-GPU runs (section "Evaluation": a mesh decomposed over
 * GPUs; per PCG iteration one halo exchange of the search direction p and the global sums of
 * the recurrence; per step one exchange of T and the sums of xRef and normFactor), emulated
 * in one cooperative launch on one GPU: every part keeps its own vectors (T and p with ghost
 * slots after the owned cells) and receives its neighbours' interface values only through
 * pushes into those slots, made right after the values are computed and made visible by the
 * barrier that ends the pass. Parts are contiguous ranges of cell labels (slabs along the
 * last axis of a naturally numbered box, the simple decomposition). The step and its
 * arithmetic are lfm_advance's FP64 step; only the order of the global sums differs. Covered:
 * FP64, orthogonal meshes, no volumetric source, no correctors (LFM_EINVAL otherwise). */
typedef struct lfm_dd lfm_dd;
typedef struct {
  int32_t first_label;  /* first cell label of the part */
  int32_t n_owned;      /* cells it owns (labels first_label ..) */
  int32_t n_ghost;      /* distinct outside neighbours it reads (its ghost slots) */
  int32_t n_send;       /* (interface cell, receiving part, ghost slot) triples it pushes */
} lfm_dd_counts;

/* Plan of part `part` of the decomposition of an LDU mesh (owner < neighbour) into n_parts
 * label ranges, on the host (no GPU): counts, and when the arrays are not NULL, the ghost
 * labels [n_ghost] (ascending) and the pushes [n_send] (source local id ascending, receiving
 * part, ghost slot in it). Call once with NULL arrays to size them. LFM_EINVAL for bad
 * sizes or faces. */
int lfm_dd_plan(int32_t n_cells, int32_t n_faces, const int32_t *owner, const int32_t *neighbour, int32_t n_parts,
                int32_t part, lfm_dd_counts *counts, int32_t *ghost_label, int32_t *send_src, int32_t *send_part,
                int32_t *send_slot);

/* Decomposes the configured case `ctx` (uploaded, FP64) into n_parts parts on ctx's device;
 * the parts start from ctx's current field and take ctx's coefficients, boundary conditions,
 * time step and solver controls at every advance (set them on ctx). Allocates the parts'
 * device memory (library-owned, freed by lfm_dd_destroy). n_parts in [1, co-resident CTAs of
 * the kernel]. ctx must outlive the decomposition and stay idle while it advances. */
int lfm_dd_create(lfm_dd **out, lfm_ctx *ctx, int32_t n_parts);
/* Counts of part `part`. */
int lfm_dd_part_counts(lfm_dd *dd, int32_t part, lfm_dd_counts *counts);
/* Field T[n_cells] (host, by label) into the parts / out of the parts. Synchronous. */
int lfm_dd_set_field(lfm_dd *dd, const double *T);
int lfm_dd_get_field(lfm_dd *dd, double *T);
/* n_steps (<= 1024) implicit steps of the decomposed case; out (host, may be NULL) receives
 * the per-step records. Synchronises before return. */
int lfm_dd_advance(lfm_dd *dd, int32_t n_steps, lfm_step_stats *out);
int lfm_dd_destroy(lfm_dd *dd);
/* Reason for the last non-OK return (dd NULL: of a call without a decomposition). */
const char *lfm_dd_last_error(const lfm_dd *dd);

/* Face coefficients of a general mesh on the device: the linear-interpolation weights of
 * the paper's "weights" loop (section "Code Porting") and the other per-face quantities of
 * the corrected laplacian, one thread per face. Every pointer is DEVICE memory the caller
 * owns, in the layouts of lfm_mesh / lfm_geometry (vectors as x, y, z per face or cell);
 * the call enqueues on `stream` (a cudaStream_t; NULL: the legacy default stream), waits
 * for it, and allocates and frees 4 bytes of device memory. For internal face f with owner P
 * and neighbour N, from its area vector Sf and centre Cf and the cell centres C:
 *   weights[f]     = |Sf.(C_N - Cf)| / (|Sf.(Cf - C_P)| + |Sf.(C_N - Cf)|), 0.5 when that
 *                    sum is not above 1e-150 (owner weight: face value w (T_P - T_N) + T_N)
 *   magSf[f]       = |Sf|
 *   deltaCoeffs[f] = 1 / max(n.d, 0.05 |d|), n = Sf / |Sf|, d = C_N - C_P
 *   corr_vec[3f..] = n - d deltaCoeffs[f]
 * and for boundary face b of cell bface_cell[b]: bmagSf[b] = |bSf|, bdeltaCoeffs[b] =
 * 1 / |n.(bCf - C)|. Each operation is rounded on its own, left to right (no fused
 * multiply-adds). LFM_EINVAL for a negative count, a NULL array that is needed, or a cell
 * index out of [0, n_cells) (found on the device; nothing is read through it), LFM_ECUDA for
 * a failed launch; the message in lfm_last_error(NULL). */
int lfm_face_coeffs_device(int32_t n_cells, int32_t n_faces, int32_t n_bfaces, const int32_t *owner,
                           const int32_t *neighbour, const double *Sf, const double *Cf, const double *C,
                           const int32_t *bface_cell, const double *bSf, const double *bCf, double *weights,
                           double *magSf, double *deltaCoeffs, double *corr_vec, double *bmagSf,
                           double *bdeltaCoeffs, void *stream);

/* Measures the FP64 fused multiply-add rate of `device` (FMAs per second, into *fma_per_s):
 * independent FMA chains on every SM, the best of three timed launches after a warm-up.
 * It bounds the FP64 form, which issues about 14 FP64 instructions per cell and PCG
 * iteration (the PCG recurrence of section "Evaluation" in IEEE FP64) against 160 bytes, so
 * that on a part with few FP64 units the issue rate, not HBM, can set the step time. Takes
 * about 0.1 s; allocates 8 bytes of device memory and frees it. The paper has no
 * counterpart (it is measurement, not the method). LFM_EINVAL for a bad device or a NULL
 * pointer; sets lfm_last_error(NULL) on failure. */
int lfm_measure_fp64_fma_rate(int device, double *fma_per_s);

/* Destroys the context (frees library-owned device memory; never a bound workspace). */
int lfm_destroy(lfm_ctx *ctx);

/* Reason for the last non-OK return on this context (ctx may be NULL: the last error of
 * a context-free call on this thread). */
const char *lfm_last_error(const lfm_ctx *ctx);

/* ---- batched form ------------------------------------------------------------------
 * A batch runs many independent cases (uploaded, configured contexts on one device) in one
 * persistent cooperative launch. Each case becomes a job needing a team of
 * k = ceil(n_cells / (threads * cells_per_thread[class])) CTAs (class 0: < 32768 cells,
 * 1: < 262144, 2: larger); jobs are served longest-first from a device work queue, each
 * with its case's own barriers and reductions, so a case's arithmetic is the same as when
 * it runs alone (up to the summation order that its team size sets). Results (T,
 * statistics) stay in each member context. While a batch advance is pending the member
 * contexts must not be used directly. */
typedef struct lfm_batch lfm_batch;

/* Creates an empty batch on `device`, issuing work on `cuda_stream` (NULL = default). */
int lfm_batch_create(lfm_batch **out, int device, void *cuda_stream);

/* Adds an uploaded context (same device, no pending advance, in no other batch); its case
 * id is written to case_id. The context stays owned by the caller and cannot be destroyed
 * while it is a member. */
int lfm_batch_add(lfm_batch *b, lfm_ctx *ctx, int32_t *case_id);

/* Removes a case (its id may be reused by a later add). */
int lfm_batch_remove(lfm_batch *b, int32_t case_id);

/* Number of member cases. */
int lfm_batch_size(const lfm_batch *b);

/* Launch shape: threads per CTA (256 or 512) and cells per thread for the three size
 * classes (NULL keeps the current ones; defaults 512 and {4, 8, 16}). */
int lfm_batch_set_launch(lfm_batch *b, int32_t threads, const int32_t *cells_per_thread);

/* Test switch of a batch, as lfm_debug_stage_rows for a context: on != 0 (the default) lets
 * the batched kernel stream A p's matrix rows into shared memory for mixed cases of six slots
 * per cell with N a multiple of 4; 0 makes it load them into registers. Same results bit for
 * bit. */
int lfm_batch_debug_stage_rows(lfm_batch *b, int32_t on);

/* Current launch shape (ctas = CTAs of the persistent launch). */
int lfm_batch_get_launch(lfm_batch *b, int32_t *ctas, int32_t *threads, int32_t *cells_per_thread);

/* Device-side barrier wait limit for batch launches (default 10 s). */
int lfm_batch_set_barrier_timeout(lfm_batch *b, uint64_t ns);

/* Enqueues n_steps (<= 1024) steps of every member case. use_graph != 0: one step is
 * captured once into a CUDA graph (ticket reset + persistent kernel) and the graph is
 * launched n_steps times; use_graph == 0: one launch runs all n_steps. Members may mix
 * precisions; when every member runs LFM_FP64, or every member LFM_DF64 (hexahedral slot
 * width), the launch uses a kernel compiled for that precision alone (same results, less
 * code around the iteration loops). */
int lfm_batch_advance_async(lfm_batch *b, int32_t n_steps, int32_t use_graph);

/* As lfm_batch_advance_async, with a cap per case: case id runs min(n_steps, caps[id]) steps
 * of this advance (ids >= n_caps run all n_steps; caps[id] >= 0, else LFM_EINVAL). A case
 * whose cap is reached takes no further step; its team's CTAs serve the other cases' jobs
 * in the same launch. The serving form uses it to run several steps per tick while each
 * request stops at its own step count (section "Evaluation": the time loop of each case is
 * the listing's; only how many of its steps share one launch changes). */
int lfm_batch_advance_capped_async(lfm_batch *b, int32_t n_steps, int32_t use_graph, const int32_t *caps,
                                   int32_t n_caps);

/* 1 while the pending advance runs, LFM_OK when done or none pending. */
int lfm_batch_query(lfm_batch *b);

/* Waits for the pending advance; returns LFM_OK or the first failing case's status (the
 * checked build also returns LFM_EINVAL when a kernel met an index out of range; see
 * lfm_checked_build). */
int lfm_batch_finish(lfm_batch *b);

/* Status of one case in the last finished advance. */
int lfm_batch_case_status(lfm_batch *b, int32_t case_id);

/* PCG iterations of one case's last step in the last finished advance (-1: none). */
int lfm_batch_case_iters(lfm_batch *b, int32_t case_id);

/* Copies the first n per-step records of one case's last advance to host memory. */
int lfm_batch_case_stats(lfm_batch *b, int32_t case_id, lfm_step_stats *out, int32_t n);

/* Results of the last finished advance for case ids 0 .. n-1, into host arrays of n entries
 * (each may be NULL): status (LFM_ESTATE for an id with no member), steps run and PCG
 * iterations summed over those steps. One call in place of a status and iteration query per
 * case. LFM_ESTATE while an advance is pending. */
int lfm_batch_results(lfm_batch *b, int32_t *status, int32_t *steps, int32_t *iters, int32_t n);

/* Destroys the batch (the member contexts are released, not destroyed). */
int lfm_batch_destroy(lfm_batch *b);

/* Reason for the batch's last non-OK return (b may be NULL). */
const char *lfm_batch_last_error(const lfm_batch *b);

#ifdef __cplusplus
}
#endif

#endif /* LAPFOAM_H */

/*
 * oracle.c -- TEST INFRASTRUCTURE ONLY. A plain, slow, serial FP64 CPU implementation of
 * one implicit-Euler step of laplacianFoam: mesh geometry from a box specification,
 * assembly of fvm::ddt(T) - fvm::laplacian(DT, T) in LDU face-addressed form, and the
 * diagonal-preconditioned conjugate-gradient solve with the normFactor-scaled residual.
 *
 * Only the tests, the package's smoke check and the benchmark's CPU-baseline arm may load
 * this library. It shares no code, header or helper with the CUDA path: it builds the
 * mesh, the face addressing, the matrix and the solver iterates itself.
 *
 * Paper passages followed (arXiv 2507.18268):
 *   - Eq. (1) (section "The laplacianFoam application"): dT/dt - div(DT grad T) = S_T; the
 *     printed d/dT is read as d/dt and S_T = 0 (no fvOptions sources are configured).
 *   - Listing "laplacianFoam application": each time step builds
 *     TEqn = fvm::ddt(T) - fvm::laplacian(DT, T) and calls TEqn.solve().
 *   - Section "OpenFOAM": face addressing; every face has an owner cell, internal faces a
 *     neighbour; the face normal points from owner to neighbour.
 *   - Listing "First cycle in the gradf routine": the serial scatter loop over faces
 *     (owner gets +, neighbour gets the opposite contribution); the assembly and the
 *     matrix-vector product below use that same face-loop pattern.
 *   - Section "Evaluation": PCG with the diagonal preconditioner.
 * Where the paper is silent (the discretisation coefficients, the PCG recurrence and the
 * normFactor), the standard finite-volume / OpenFOAM definitions are written out from the
 * mathematics:
 *   laplacian coefficient of internal face f:   g_f = DT_f * |S_f| * deltaCoeff_f,
 *       deltaCoeff_f = 1 / |C_N - C_P| (orthogonal hexahedra)
 *   fixedValue boundary face b:   g_b = DT_b * |S_b| / |C_b - C_P|;  it adds g_b to the
 *       diagonal and g_b * T_b to the source; zeroGradient faces add nothing
 *   Euler ddt:  diag += V/dt,  source += V/dt * T_old
 *   off-diagonals: upper_f = lower_f = -g_f
 *   PCG: Jacobi preconditioner rD = 1/diag, L1 residual sum|r| / normFactor,
 *       normFactor = sum_c (|(A x)_c - s_c xRef| + |b_c - s_c xRef|) + 1e-20,
 *       s_c = row sum of A, xRef = arithmetic mean of the initial guess x;
 *       convergence: res < tol or (relTol > 0 and res < relTol * initRes); singular when
 *       |p.Ap| / normFactor < 1e-300.
 *
 * Parity status: every function here is pinned by the CPU tests (dense LU solve, closed-form
 * steady and transient solutions, matrix symmetry and row sums, energy balance, permutation
 * invariance, finite termination of CG, hand-computed two-cell normFactors -- one with unequal
 * volumes, diagonals and row sums, which fixes the unweighted mean and the row sums -- and the
 * strict '<' of the convergence test at exact ties; for the general
 * geometry, gradient and corrected laplacian see the block below; cell-field DT and sources:
 * uniform and linear interpolation, the series-conductance steady state, closed-form source
 * steps and energy balance).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORA_FIXED_VALUE 0
#define ORA_ZERO_GRADIENT 1

typedef struct {
  int32_t nx, ny, nz;
  const double *xs, *ys, *zs;  /* vertex coordinates, nx+1 / ny+1 / nz+1 entries */
  const int64_t *perm;         /* natural cell id -> label; NULL = identity */
  double DT_uniform;           /* used when the per-face arrays are NULL */
  const double *DTx, *DTy, *DTz;
} ora_box;

typedef struct {
  int32_t iters, converged, singular, nonfinite;
  double init_res, final_res, norm_factor;
} ora_stats;

/* ------------------------------------------------------------------------------------ */
/* Mesh from the box specification                                                       */
/* ------------------------------------------------------------------------------------ */

void ora_box_counts(const ora_box *b, int64_t *n_cells, int64_t *n_faces, int64_t *n_bfaces) {
  int64_t nx = b->nx, ny = b->ny, nz = b->nz;
  *n_cells = nx * ny * nz;
  *n_faces = (nx - 1) * ny * nz + nx * (ny - 1) * nz + nx * ny * (nz - 1);
  *n_bfaces = 2 * (ny * nz + nx * nz + nx * ny);
}

typedef struct {
  int32_t own, nei;
  double magSf, delta, DT;
} ora_face;

static int face_cmp(const void *a, const void *b) {
  const ora_face *fa = (const ora_face *)a, *fb = (const ora_face *)b;
  if (fa->own != fb->own) return fa->own < fb->own ? -1 : 1;
  if (fa->nei != fb->nei) return fa->nei < fb->nei ? -1 : 1;
  return 0;
}

static int64_t label_of(const ora_box *b, int64_t i, int64_t j, int64_t k) {
  int64_t nat = i + (int64_t)b->nx * (j + (int64_t)b->ny * k);
  return b->perm ? b->perm[nat] : nat;
}

static double face_dt(const double *arr, double uniform, int64_t idx) {
  return arr ? arr[idx] : uniform;
}

/* Cell-centre coordinate and width of cell i along an axis with vertices v[0..n]. */
static double centre(const double *v, int64_t i) { return 0.5 * (v[i] + v[i + 1]); }
static double width(const double *v, int64_t i) { return v[i + 1] - v[i]; }

/*
 * Fills the LDU mesh: internal faces in upper-triangular order (sorted by owner, then
 * neighbour, owner < neighbour), boundary faces grouped by patch x0,x1,y0,y1,z0,z1.
 * Returns 0, or -1 when memory runs out.
 */
int ora_box_mesh(const ora_box *b, int32_t *owner, int32_t *neighbour, double *V, double *magSf,
                 double *delta, double *DTf, int32_t *bcell, int32_t *bpatch, double *bmagSf,
                 double *bdelta, double *DTb) {
  int64_t nx = b->nx, ny = b->ny, nz = b->nz;
  int64_t N, F, NB;
  ora_box_counts(b, &N, &F, &NB);
  ora_face *faces = (ora_face *)malloc(sizeof(ora_face) * (size_t)(F > 0 ? F : 1));
  if (!faces) return -1;

  for (int64_t k = 0; k < nz; ++k)
    for (int64_t j = 0; j < ny; ++j)
      for (int64_t i = 0; i < nx; ++i)
        V[label_of(b, i, j, k)] = width(b->xs, i) * width(b->ys, j) * width(b->zs, k);

  int64_t nf = 0;
  for (int64_t k = 0; k < nz; ++k)
    for (int64_t j = 0; j < ny; ++j)
      for (int64_t i = 0; i < nx; ++i) {
        int64_t P = label_of(b, i, j, k);
        if (i + 1 < nx) { /* x-normal face between (i,j,k) and (i+1,j,k) */
          int64_t Q = label_of(b, i + 1, j, k);
          ora_face *f = &faces[nf++];
          f->own = (int32_t)(P < Q ? P : Q);
          f->nei = (int32_t)(P < Q ? Q : P);
          f->magSf = width(b->ys, j) * width(b->zs, k);
          f->delta = 1.0 / (centre(b->xs, i + 1) - centre(b->xs, i));
          f->DT = face_dt(b->DTx, b->DT_uniform, (k * ny + j) * (nx + 1) + (i + 1));
        }
        if (j + 1 < ny) { /* y-normal face */
          int64_t Q = label_of(b, i, j + 1, k);
          ora_face *f = &faces[nf++];
          f->own = (int32_t)(P < Q ? P : Q);
          f->nei = (int32_t)(P < Q ? Q : P);
          f->magSf = width(b->xs, i) * width(b->zs, k);
          f->delta = 1.0 / (centre(b->ys, j + 1) - centre(b->ys, j));
          f->DT = face_dt(b->DTy, b->DT_uniform, (k * (ny + 1) + (j + 1)) * nx + i);
        }
        if (k + 1 < nz) { /* z-normal face */
          int64_t Q = label_of(b, i, j, k + 1);
          ora_face *f = &faces[nf++];
          f->own = (int32_t)(P < Q ? P : Q);
          f->nei = (int32_t)(P < Q ? Q : P);
          f->magSf = width(b->xs, i) * width(b->ys, j);
          f->delta = 1.0 / (centre(b->zs, k + 1) - centre(b->zs, k));
          f->DT = face_dt(b->DTz, b->DT_uniform, ((k + 1) * ny + j) * nx + i);
        }
      }
  qsort(faces, (size_t)nf, sizeof(ora_face), face_cmp);
  for (int64_t f = 0; f < nf; ++f) {
    owner[f] = faces[f].own;
    neighbour[f] = faces[f].nei;
    magSf[f] = faces[f].magSf;
    delta[f] = faces[f].delta;
    DTf[f] = faces[f].DT;
  }
  free(faces);

  int64_t nb = 0;
  for (int side = 0; side < 2; ++side) { /* patches x0, x1 */
    int64_t i = side ? nx - 1 : 0, ip = side ? nx : 0;
    double facex = b->xs[ip];
    for (int64_t k = 0; k < nz; ++k)
      for (int64_t j = 0; j < ny; ++j, ++nb) {
        bcell[nb] = (int32_t)label_of(b, i, j, k);
        bpatch[nb] = side;
        bmagSf[nb] = width(b->ys, j) * width(b->zs, k);
        bdelta[nb] = 1.0 / fabs(facex - centre(b->xs, i));
        DTb[nb] = face_dt(b->DTx, b->DT_uniform, (k * ny + j) * (nx + 1) + ip);
      }
  }
  for (int side = 0; side < 2; ++side) { /* patches y0, y1 */
    int64_t j = side ? ny - 1 : 0, jp = side ? ny : 0;
    double facey = b->ys[jp];
    for (int64_t k = 0; k < nz; ++k)
      for (int64_t i = 0; i < nx; ++i, ++nb) {
        bcell[nb] = (int32_t)label_of(b, i, j, k);
        bpatch[nb] = 2 + side;
        bmagSf[nb] = width(b->xs, i) * width(b->zs, k);
        bdelta[nb] = 1.0 / fabs(facey - centre(b->ys, j));
        DTb[nb] = face_dt(b->DTy, b->DT_uniform, (k * (ny + 1) + jp) * nx + i);
      }
  }
  for (int side = 0; side < 2; ++side) { /* patches z0, z1 */
    int64_t k = side ? nz - 1 : 0, kp = side ? nz : 0;
    double facez = b->zs[kp];
    for (int64_t j = 0; j < ny; ++j)
      for (int64_t i = 0; i < nx; ++i, ++nb) {
        bcell[nb] = (int32_t)label_of(b, i, j, k);
        bpatch[nb] = 4 + side;
        bmagSf[nb] = width(b->xs, i) * width(b->ys, j);
        bdelta[nb] = 1.0 / fabs(facez - centre(b->zs, k));
        DTb[nb] = face_dt(b->DTz, b->DT_uniform, (kp * ny + j) * nx + i);
      }
  }
  return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Assembly: fvm::ddt(T) - fvm::laplacian(DT, T), scatter over faces                      */
/* ------------------------------------------------------------------------------------ */

/* Su, Sp (may be NULL): the source S_T = Su + Sp T of Eq. (1) per unit volume (fvOptions);
 * on the right-hand side of the equation it adds V Su to the source and -V Sp to the
 * diagonal. */
void ora_assemble(int64_t N, int64_t F, const int32_t *owner, const int32_t *neighbour,
                  const double *V, const double *magSf, const double *delta, const double *DTf,
                  int64_t NB, const int32_t *bcell, const int32_t *btype, const double *bvalue,
                  const double *bmagSf, const double *bdelta, const double *DTb, double dt,
                  const double *T_old, const double *Su, const double *Sp, double *diag, double *upper,
                  double *source) {
  for (int64_t c = 0; c < N; ++c) {
    diag[c] = 0.0;
    source[c] = 0.0;
  }
  /* laplacian: each internal face couples its owner and neighbour */
  for (int64_t f = 0; f < F; ++f) {
    double g = DTf[f] * magSf[f] * delta[f];
    upper[f] = -g;
    diag[owner[f]] += g;
    diag[neighbour[f]] += g;
  }
  /* boundary: fixedValue faces add g_b to the diagonal and g_b*T_b to the source */
  for (int64_t b = 0; b < NB; ++b) {
    if (btype[b] != ORA_FIXED_VALUE) continue;
    double gb = DTb[b] * bmagSf[b] * bdelta[b];
    diag[bcell[b]] += gb;
    source[bcell[b]] += gb * bvalue[b];
  }
  /* Euler implicit ddt */
  for (int64_t c = 0; c < N; ++c) {
    double vdt = V[c] / dt;
    diag[c] += vdt;
    source[c] += vdt * T_old[c];
  }
  /* volumetric source S_T = Su + Sp T */
  for (int64_t c = 0; c < N; ++c) {
    if (Sp) diag[c] -= V[c] * Sp[c];
    if (Su) source[c] += V[c] * Su[c];
  }
}

/*
 * Diffusivity given as a cell field (a volScalarField): internal faces take the linear
 * interpolate in the form of the paper's listing "dotInterpolate loop",
 * w_f (DT_P - DT_N) + DT_N, boundary faces the value of their cell.
 */
void ora_cell_dt_to_faces(int64_t F, int64_t NB, const int32_t *owner, const int32_t *neighbour,
                          const double *w, const int32_t *bcell, const double *DTc, double *DTf, double *DTb) {
  for (int64_t f = 0; f < F; ++f) DTf[f] = w[f] * (DTc[owner[f]] - DTc[neighbour[f]]) + DTc[neighbour[f]];
  for (int64_t b = 0; b < NB; ++b) DTb[b] = DTc[bcell[b]];
}

/* y = A x with A in LDU form (lower = upper), scatter over faces. */
void ora_amul(int64_t N, int64_t F, const int32_t *owner, const int32_t *neighbour,
              const double *diag, const double *upper, const double *x, double *y) {
  for (int64_t c = 0; c < N; ++c) y[c] = diag[c] * x[c];
  for (int64_t f = 0; f < F; ++f) {
    y[owner[f]] += upper[f] * x[neighbour[f]];
    y[neighbour[f]] += upper[f] * x[owner[f]];
  }
}

/* ------------------------------------------------------------------------------------ */
/* Diagonal-preconditioned CG with the normFactor residual                               */
/* ------------------------------------------------------------------------------------ */

static int is_converged(double res, double init_res, double tol, double rel_tol) {
  return res < tol || (rel_tol > 0.0 && res < rel_tol * init_res);
}

/*
 * Solves A psi = source starting from psi. trace_p (optional) receives the search
 * direction of each of the first max_trace iterations (N doubles each).
 * Returns 0, or -1 when memory runs out.
 */
int ora_pcg(int64_t N, int64_t F, const int32_t *owner, const int32_t *neighbour,
            const double *diag, const double *upper, const double *source, double *psi,
            double tol, double rel_tol, int32_t max_iter, int32_t min_iter, ora_stats *st,
            double *trace_p, int32_t max_trace) {
  double *wA = (double *)malloc(sizeof(double) * (size_t)N);
  double *rA = (double *)malloc(sizeof(double) * (size_t)N);
  double *pA = (double *)malloc(sizeof(double) * (size_t)N);
  double *sumA = (double *)malloc(sizeof(double) * (size_t)N);
  double *rD = (double *)malloc(sizeof(double) * (size_t)N);
  if (!wA || !rA || !pA || !sumA || !rD) {
    free(wA); free(rA); free(pA); free(sumA); free(rD);
    return -1;
  }
  memset(st, 0, sizeof(*st));

  /* initial residual */
  ora_amul(N, F, owner, neighbour, diag, upper, psi, wA);
  for (int64_t c = 0; c < N; ++c) rA[c] = source[c] - wA[c];

  /* normFactor: row sums s_c and the mean of the initial guess */
  for (int64_t c = 0; c < N; ++c) sumA[c] = diag[c];
  for (int64_t f = 0; f < F; ++f) {
    sumA[owner[f]] += upper[f];
    sumA[neighbour[f]] += upper[f];
  }
  double xsum = 0.0;
  for (int64_t c = 0; c < N; ++c) xsum += psi[c];
  double xRef = xsum / (double)N;
  double nf = 0.0;
  for (int64_t c = 0; c < N; ++c) {
    double pAc = sumA[c] * xRef;
    nf += fabs(wA[c] - pAc) + fabs(source[c] - pAc);
  }
  nf += 1e-20;
  st->norm_factor = nf;

  double rsum = 0.0;
  for (int64_t c = 0; c < N; ++c) rsum += fabs(rA[c]);
  st->init_res = rsum / nf;
  st->final_res = st->init_res;

  for (int64_t c = 0; c < N; ++c) rD[c] = 1.0 / diag[c];

  int32_t n_iter = 0;
  if (min_iter > 0 || !is_converged(st->final_res, st->init_res, tol, rel_tol)) {
    double rho_old = 0.0;
    do {
      /* precondition: w = rD r (stored in wA) */
      for (int64_t c = 0; c < N; ++c) wA[c] = rD[c] * rA[c];
      double rho = 0.0;
      for (int64_t c = 0; c < N; ++c) rho += wA[c] * rA[c];
      if (n_iter == 0) {
        for (int64_t c = 0; c < N; ++c) pA[c] = wA[c];
      } else {
        double beta = rho / rho_old;
        for (int64_t c = 0; c < N; ++c) pA[c] = wA[c] + beta * pA[c];
      }
      if (trace_p && n_iter < max_trace) memcpy(trace_p + (size_t)n_iter * (size_t)N, pA, sizeof(double) * (size_t)N);
      /* q = A p (stored in wA) */
      ora_amul(N, F, owner, neighbour, diag, upper, pA, wA);
      double sigma = 0.0;
      for (int64_t c = 0; c < N; ++c) sigma += wA[c] * pA[c];
      if (fabs(sigma) / nf < 1e-300) {
        st->singular = 1;
        break;
      }
      double alpha = rho / sigma;
      for (int64_t c = 0; c < N; ++c) {
        psi[c] += alpha * pA[c];
        rA[c] -= alpha * wA[c];
      }
      rsum = 0.0;
      for (int64_t c = 0; c < N; ++c) rsum += fabs(rA[c]);
      st->final_res = rsum / nf;
      rho_old = rho;
      if (!isfinite(st->final_res)) {
        st->nonfinite = 1;
        ++n_iter;
        break;
      }
    } while ((++n_iter < max_iter && !is_converged(st->final_res, st->init_res, tol, rel_tol)) ||
             n_iter < min_iter);
  }
  st->iters = n_iter;
  st->converged = is_converged(st->final_res, st->init_res, tol, rel_tol);
  free(wA); free(rA); free(pA); free(sumA); free(rD);
  return 0;
}

/*
 * n_steps implicit-Euler steps: T_old <- T, assemble, PCG from T_old, T <- solution.
 * stats receives one record per step. Returns 0, or -1 when memory runs out.
 */
int ora_advance(int64_t N, int64_t F, const int32_t *owner, const int32_t *neighbour,
                const double *V, const double *magSf, const double *delta, const double *DTf,
                int64_t NB, const int32_t *bcell, const int32_t *btype, const double *bvalue,
                const double *bmagSf, const double *bdelta, const double *DTb, double dt,
                int32_t n_steps, double tol, double rel_tol, int32_t max_iter, int32_t min_iter,
                const double *Su, const double *Sp, double *T, ora_stats *stats) {
  double *diag = (double *)malloc(sizeof(double) * (size_t)N);
  double *upper = (double *)malloc(sizeof(double) * (size_t)(F > 0 ? F : 1));
  double *source = (double *)malloc(sizeof(double) * (size_t)N);
  double *T_old = (double *)malloc(sizeof(double) * (size_t)N);
  int rc = 0;
  if (!diag || !upper || !source || !T_old) rc = -1;
  for (int32_t s = 0; s < n_steps && rc == 0; ++s) {
    memcpy(T_old, T, sizeof(double) * (size_t)N);
    ora_assemble(N, F, owner, neighbour, V, magSf, delta, DTf, NB, bcell, btype, bvalue, bmagSf,
                 bdelta, DTb, dt, T_old, Su, Sp, diag, upper, source);
    rc = ora_pcg(N, F, owner, neighbour, diag, upper, source, T, tol, rel_tol, max_iter, min_iter,
                 &stats[s], NULL, 0);
  }
  free(diag); free(upper); free(source); free(T_old);
  return rc;
}

/* Boundary-face values of the field: fixedValue -> the set value, zeroGradient -> the
 * value of the face's cell. */
void ora_boundary_values(int64_t NB, const int32_t *bcell, const int32_t *btype,
                         const double *bvalue, const double *T, double *Tb) {
  for (int64_t b = 0; b < NB; ++b)
    Tb[b] = btype[b] == ORA_FIXED_VALUE ? bvalue[b] : T[bcell[b]];
}

/* ==================================================================================== */
/* General hexahedral meshes: geometry, Gauss linear gradient, non-orthogonal correction */
/* ==================================================================================== */
/*
 * Paper passages followed: the listings "weights parallel loop" (interpolation weights),
 * "dotInterpolate loop" (face value lambda*(v_P - v_N) + v_N), "First cycle in the gradf
 * routine" and "Second cycle gradient" (Gauss sum over internal and boundary faces), "Field
 * division" (division by the cell volume) and "CorrectBoundaryConditions" (boundary gradient
 * normal component replaced by the patch snGrad); section "Code Porting".
 * Where the paper is silent, the standard OpenFOAM definitions are written out:
 *   face centre / area vector: triangle fan about the average of the face points; each
 *     triangle (p_i, p_i+1, c) contributes n_i = (p_i+1 - p_i) x (c - p_i) to the area
 *     (1/2 sum n_i) and its centroid, weighted by |n_i|, to the face centre;
 *   cell centre / volume: pyramids from each face to the average of the cell's face centres,
 *     volume 1/3 Sf.(Cf - c_est), centroid 3/4 Cf + 1/4 c_est;
 *   nonOrthDeltaCoeff_f = 1 / max(n.d, 0.05 |d|), d = C_N - C_P, n = Sf/|Sf|;
 *   correction vector k_f = n - d * nonOrthDeltaCoeff_f (zero on boundary faces);
 *   boundary deltaCoeff = 1 / |n.(Cf - C_P)| (patch-normal distance);
 *   corrected laplacian: implicit coefficient DT |Sf| nonOrthDeltaCoeff, explicit flux
 *     DT |Sf| k_f . (w_f (G_P - G_N) + G_N) with G the Gauss linear gradient of the current
 *     T; it enters the source as V * div(flux) (surface integral / V, times V);
 *   nNonOrthCorr extra assemble-and-solve passes per time step, each with the correction
 *     from the latest T and the ddt term from T at the start of the step.
 * Vertex (i, j, k) of a box with nx x ny x nz cells is pts[3 * (i + (nx+1) * (j + (ny+1) k))].
 * Cells carry natural labels i + nx (j + ny k); internal faces come cell by cell in the order
 * +x, +y, +z (upper-triangular order), boundary faces by patch as for the rectilinear box.
 * Face points run so that the area vector points from owner to neighbour (outward on the
 * boundary).
 */

typedef struct {
  int32_t nx, ny, nz;
  const double *pts;
} ora_hex;

static const double *hex_pt(const ora_hex *h, int64_t i, int64_t j, int64_t k) {
  return h->pts + 3 * (i + (int64_t)(h->nx + 1) * (j + (int64_t)(h->ny + 1) * k));
}

static void v_sub(const double *a, const double *b, double *o) {
  o[0] = a[0] - b[0];
  o[1] = a[1] - b[1];
  o[2] = a[2] - b[2];
}
static void v_cross(const double *a, const double *b, double *o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}
static double v_dot(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static double v_mag(const double *a) { return sqrt(v_dot(a, a)); }

/* Centre and area vector of the quadrilateral face q[0..3] (triangle fan). */
static void quad_geometry(const double *q[4], double *Cf, double *Sf) {
  double fc[3] = {q[0][0], q[0][1], q[0][2]};
  for (int p = 1; p < 4; ++p)
    for (int d = 0; d < 3; ++d) fc[d] += q[p][d];
  for (int d = 0; d < 3; ++d) fc[d] /= 4.0;
  double sumN[3] = {0, 0, 0}, sumA = 0.0, sumAc[3] = {0, 0, 0};
  for (int p = 0; p < 4; ++p) {
    const double *a = q[p], *b = q[(p + 1) % 4];
    double e[3], t[3], n[3];
    v_sub(b, a, e);
    v_sub(fc, a, t);
    v_cross(e, t, n);
    double mag = v_mag(n);
    for (int d = 0; d < 3; ++d) {
      double c = a[d] + b[d] + fc[d];
      sumN[d] += n[d];
      sumAc[d] += mag * c;
    }
    sumA += mag;
  }
  for (int d = 0; d < 3; ++d) {
    Cf[d] = sumA > 1e-300 ? (1.0 / 3.0) * sumAc[d] / sumA : fc[d];
    Sf[d] = 0.5 * sumN[d];
  }
}

void ora_hex_counts(const ora_hex *h, int64_t *n_cells, int64_t *n_faces, int64_t *n_bfaces) {
  int64_t nx = h->nx, ny = h->ny, nz = h->nz;
  *n_cells = nx * ny * nz;
  *n_faces = (nx - 1) * ny * nz + nx * (ny - 1) * nz + nx * ny * (nz - 1);
  *n_bfaces = 2 * (ny * nz + nx * nz + nx * ny);
}

/*
 * Topology and geometry of the hexahedral mesh: owner/neighbour, face area vectors and
 * centres (internal Sf/Cf [3F], boundary bSf/bCf [3NB]), boundary cells and patches, cell
 * volumes V [N] and centres C [3N]. Returns 0, or -1 when memory runs out.
 */
int ora_hex_mesh(const ora_hex *h, int32_t *owner, int32_t *neighbour, double *Sf, double *Cf,
                 int32_t *bcell, int32_t *bpatch, double *bSf, double *bCf, double *V, double *C) {
  int64_t nx = h->nx, ny = h->ny, nz = h->nz;
  int64_t N, F, NB;
  ora_hex_counts(h, &N, &F, &NB);
  int64_t nf = 0;
  for (int64_t k = 0; k < nz; ++k)
    for (int64_t j = 0; j < ny; ++j)
      for (int64_t i = 0; i < nx; ++i) {
        int64_t P = i + nx * (j + ny * k);
        if (i + 1 < nx) { /* +x face: points at i+1, order (j,k) (j+1,k) (j+1,k+1) (j,k+1) */
          const double *q[4] = {hex_pt(h, i + 1, j, k), hex_pt(h, i + 1, j + 1, k), hex_pt(h, i + 1, j + 1, k + 1),
                                hex_pt(h, i + 1, j, k + 1)};
          owner[nf] = (int32_t)P;
          neighbour[nf] = (int32_t)(P + 1);
          quad_geometry(q, Cf + 3 * nf, Sf + 3 * nf);
          ++nf;
        }
        if (j + 1 < ny) { /* +y face: points at j+1, order (i,k) (i,k+1) (i+1,k+1) (i+1,k) */
          const double *q[4] = {hex_pt(h, i, j + 1, k), hex_pt(h, i, j + 1, k + 1), hex_pt(h, i + 1, j + 1, k + 1),
                                hex_pt(h, i + 1, j + 1, k)};
          owner[nf] = (int32_t)P;
          neighbour[nf] = (int32_t)(P + nx);
          quad_geometry(q, Cf + 3 * nf, Sf + 3 * nf);
          ++nf;
        }
        if (k + 1 < nz) { /* +z face: points at k+1, order (i,j) (i+1,j) (i+1,j+1) (i,j+1) */
          const double *q[4] = {hex_pt(h, i, j, k + 1), hex_pt(h, i + 1, j, k + 1), hex_pt(h, i + 1, j + 1, k + 1),
                                hex_pt(h, i, j + 1, k + 1)};
          owner[nf] = (int32_t)P;
          neighbour[nf] = (int32_t)(P + nx * ny);
          quad_geometry(q, Cf + 3 * nf, Sf + 3 * nf);
          ++nf;
        }
      }
  int64_t nb = 0;
  for (int side = 0; side < 2; ++side) { /* x0 (outward -x), x1 (+x) */
    int64_t i = side ? nx - 1 : 0, ip = side ? nx : 0;
    for (int64_t k = 0; k < nz; ++k)
      for (int64_t j = 0; j < ny; ++j, ++nb) {
        const double *q0[4] = {hex_pt(h, ip, j, k), hex_pt(h, ip, j, k + 1), hex_pt(h, ip, j + 1, k + 1),
                               hex_pt(h, ip, j + 1, k)};
        const double *q1[4] = {hex_pt(h, ip, j, k), hex_pt(h, ip, j + 1, k), hex_pt(h, ip, j + 1, k + 1),
                               hex_pt(h, ip, j, k + 1)};
        bcell[nb] = (int32_t)(i + nx * (j + ny * k));
        bpatch[nb] = side;
        quad_geometry(side ? q1 : q0, bCf + 3 * nb, bSf + 3 * nb);
      }
  }
  for (int side = 0; side < 2; ++side) { /* y0 (-y), y1 (+y) */
    int64_t j = side ? ny - 1 : 0, jp = side ? ny : 0;
    for (int64_t k = 0; k < nz; ++k)
      for (int64_t i = 0; i < nx; ++i, ++nb) {
        const double *q0[4] = {hex_pt(h, i, jp, k), hex_pt(h, i + 1, jp, k), hex_pt(h, i + 1, jp, k + 1),
                               hex_pt(h, i, jp, k + 1)};
        const double *q1[4] = {hex_pt(h, i, jp, k), hex_pt(h, i, jp, k + 1), hex_pt(h, i + 1, jp, k + 1),
                               hex_pt(h, i + 1, jp, k)};
        bcell[nb] = (int32_t)(i + nx * (j + ny * k));
        bpatch[nb] = 2 + side;
        quad_geometry(side ? q1 : q0, bCf + 3 * nb, bSf + 3 * nb);
      }
  }
  for (int side = 0; side < 2; ++side) { /* z0 (-z), z1 (+z) */
    int64_t k = side ? nz - 1 : 0, kp = side ? nz : 0;
    for (int64_t j = 0; j < ny; ++j)
      for (int64_t i = 0; i < nx; ++i, ++nb) {
        const double *q0[4] = {hex_pt(h, i, j, kp), hex_pt(h, i, j + 1, kp), hex_pt(h, i + 1, j + 1, kp),
                               hex_pt(h, i + 1, j, kp)};
        const double *q1[4] = {hex_pt(h, i, j, kp), hex_pt(h, i + 1, j, kp), hex_pt(h, i + 1, j + 1, kp),
                               hex_pt(h, i, j + 1, kp)};
        bcell[nb] = (int32_t)(i + nx * (j + ny * k));
        bpatch[nb] = 4 + side;
        quad_geometry(side ? q1 : q0, bCf + 3 * nb, bSf + 3 * nb);
      }
  }

  /* cell centres and volumes: pyramids about the average of the cell's face centres */
  double *cEst = (double *)calloc((size_t)(3 * N), sizeof(double));
  int32_t *nCF = (int32_t *)calloc((size_t)N, sizeof(int32_t));
  double *vol = (double *)calloc((size_t)N, sizeof(double));
  if (!cEst || !nCF || !vol) {
    free(cEst); free(nCF); free(vol);
    return -1;
  }
  for (int64_t f = 0; f < F; ++f) {
    for (int d = 0; d < 3; ++d) {
      cEst[3 * owner[f] + d] += Cf[3 * f + d];
      cEst[3 * neighbour[f] + d] += Cf[3 * f + d];
    }
    ++nCF[owner[f]];
    ++nCF[neighbour[f]];
  }
  for (int64_t b = 0; b < NB; ++b) {
    for (int d = 0; d < 3; ++d) cEst[3 * bcell[b] + d] += bCf[3 * b + d];
    ++nCF[bcell[b]];
  }
  for (int64_t c = 0; c < N; ++c)
    for (int d = 0; d < 3; ++d) cEst[3 * c + d] /= (double)nCF[c];
  for (int64_t c = 0; c < 3 * N; ++c) C[c] = 0.0;
  for (int64_t f = 0; f < F; ++f) {
    double t[3];
    int64_t P = owner[f], Q = neighbour[f];
    v_sub(Cf + 3 * f, cEst + 3 * P, t);
    double pv = fmax(v_dot(Sf + 3 * f, t), 1e-300);
    for (int d = 0; d < 3; ++d) C[3 * P + d] += pv * (0.75 * Cf[3 * f + d] + 0.25 * cEst[3 * P + d]);
    vol[P] += pv;
    v_sub(cEst + 3 * Q, Cf + 3 * f, t);
    pv = fmax(v_dot(Sf + 3 * f, t), 1e-300);
    for (int d = 0; d < 3; ++d) C[3 * Q + d] += pv * (0.75 * Cf[3 * f + d] + 0.25 * cEst[3 * Q + d]);
    vol[Q] += pv;
  }
  for (int64_t b = 0; b < NB; ++b) {
    double t[3];
    int64_t P = bcell[b];
    v_sub(bCf + 3 * b, cEst + 3 * P, t);
    double pv = fmax(v_dot(bSf + 3 * b, t), 1e-300);
    for (int d = 0; d < 3; ++d) C[3 * P + d] += pv * (0.75 * bCf[3 * b + d] + 0.25 * cEst[3 * P + d]);
    vol[P] += pv;
  }
  for (int64_t c = 0; c < N; ++c) {
    for (int d = 0; d < 3; ++d) C[3 * c + d] /= vol[c];
    V[c] = vol[c] / 3.0;
  }
  free(cEst); free(nCF); free(vol);
  return 0;
}

/*
 * Interpolation weights, |Sf|, nonOrthDeltaCoeffs and correction vectors of the internal
 * faces; |Sf| and deltaCoeffs (patch-normal distance) of the boundary faces.
 */
void ora_hex_coeffs(int64_t F, int64_t NB, const int32_t *owner, const int32_t *neighbour, const double *Sf,
                    const double *Cf, const double *C, const int32_t *bcell, const double *bSf,
                    const double *bCf, double *w, double *magSf, double *nonOrthDelta, double *corr,
                    double *bmagSf, double *bdelta) {
  for (int64_t f = 0; f < F; ++f) {
    const double *s = Sf + 3 * f, *cf = Cf + 3 * f, *cp = C + 3 * owner[f], *cn = C + 3 * neighbour[f];
    double a[3], b[3];
    v_sub(cf, cp, a);
    v_sub(cn, cf, b);
    double SfdOwn = fabs(v_dot(s, a)), SfdNei = fabs(v_dot(s, b));
    w[f] = fabs(SfdOwn + SfdNei) > 1e-150 ? SfdNei / (SfdOwn + SfdNei) : 0.5;
    double mag = v_mag(s), n[3], d[3];
    magSf[f] = mag;
    for (int k = 0; k < 3; ++k) n[k] = s[k] / mag;
    v_sub(cn, cp, d);
    double nd = fmax(v_dot(n, d), 0.05 * v_mag(d));
    nonOrthDelta[f] = 1.0 / nd;
    for (int k = 0; k < 3; ++k) corr[3 * f + k] = n[k] - d[k] * nonOrthDelta[f];
  }
  for (int64_t b = 0; b < NB; ++b) {
    const double *s = bSf + 3 * b;
    double mag = v_mag(s), n[3], t[3];
    bmagSf[b] = mag;
    for (int k = 0; k < 3; ++k) n[k] = s[k] / mag;
    v_sub(bCf + 3 * b, C + 3 * bcell[b], t);
    bdelta[b] = 1.0 / fabs(v_dot(n, t));
  }
}

/*
 * Gauss linear gradient of T (cells, [3N]) following the paper's passes: face values by
 * linear interpolation (internal) or the boundary values Tb; the Gauss sum as the serial
 * scatter loop over internal faces (owner +, neighbour -) and the boundary loop; division
 * by the cell volume. Returns 0, or -1 when memory runs out.
 */
int ora_gauss_grad(int64_t N, int64_t F, int64_t NB, const int32_t *owner, const int32_t *neighbour,
                   const double *Sf, const double *w, const double *V, const int32_t *bcell, const double *bSf,
                   const double *Tb, const double *T, double *G) {
  double *Tf = (double *)malloc(sizeof(double) * (size_t)(F > 0 ? F : 1));
  if (!Tf) return -1;
  for (int64_t f = 0; f < F; ++f) Tf[f] = w[f] * (T[owner[f]] - T[neighbour[f]]) + T[neighbour[f]];
  for (int64_t c = 0; c < 3 * N; ++c) G[c] = 0.0;
  for (int64_t f = 0; f < F; ++f)
    for (int d = 0; d < 3; ++d) {
      double v = Sf[3 * f + d] * Tf[f];
      G[3 * owner[f] + d] += v;
      G[3 * neighbour[f] + d] -= v;
    }
  for (int64_t b = 0; b < NB; ++b)
    for (int d = 0; d < 3; ++d) G[3 * bcell[b] + d] += bSf[3 * b + d] * Tb[b];
  for (int64_t c = 0; c < N; ++c)
    for (int d = 0; d < 3; ++d) G[3 * c + d] /= V[c];
  free(Tf);
  return 0;
}

/*
 * Boundary values of the gradient [3NB]: the adjacent cell's gradient with its normal
 * component replaced by the patch snGrad (fixedValue: (T_b - T_P) * deltaCoeff;
 * zeroGradient: 0).
 */
void ora_grad_boundary(int64_t NB, const int32_t *bcell, const double *bSf, const double *bdelta,
                       const int32_t *btype, const double *bvalue, const double *T, const double *G,
                       double *Gb) {
  for (int64_t b = 0; b < NB; ++b) {
    const double *s = bSf + 3 * b, *g = G + 3 * bcell[b];
    double mag = v_mag(s), n[3];
    for (int k = 0; k < 3; ++k) n[k] = s[k] / mag;
    double sn = btype[b] == ORA_FIXED_VALUE ? (bvalue[b] - T[bcell[b]]) * bdelta[b] : 0.0;
    double gn = v_dot(n, g);
    for (int k = 0; k < 3; ++k) Gb[3 * b + k] = g[k] + n[k] * (sn - gn);
  }
}

/*
 * n_steps implicit-Euler steps with the corrected laplacian: per step 1 + n_corr passes of
 * (Gauss gradient of the current T -> correction flux -> assembly with the ddt term from
 * the step's starting T -> PCG from the current T). stats receives one record per step:
 * iterations summed over the passes, the first pass's initial residual and normFactor, the
 * last pass's final residual and convergence. Returns 0, or -1 when memory runs out.
 */
int ora_advance_corrected(int64_t N, int64_t F, const int32_t *owner, const int32_t *neighbour,
                          const double *V, const double *magSf, const double *nonOrthDelta,
                          const double *DTf, const double *Sf, const double *w, const double *corr,
                          int64_t NB, const int32_t *bcell, const int32_t *btype, const double *bvalue,
                          const double *bmagSf, const double *bdelta, const double *DTb, const double *bSf,
                          double dt, int32_t n_steps, int32_t n_corr, double tol, double rel_tol,
                          int32_t max_iter, int32_t min_iter, const double *Su, const double *Sp, double *T,
                          ora_stats *stats) {
  double *diag = (double *)malloc(sizeof(double) * (size_t)N);
  double *upper = (double *)malloc(sizeof(double) * (size_t)(F > 0 ? F : 1));
  double *source = (double *)malloc(sizeof(double) * (size_t)N);
  double *T_old = (double *)malloc(sizeof(double) * (size_t)N);
  double *G = (double *)malloc(sizeof(double) * (size_t)(3 * N));
  double *Tb = (double *)malloc(sizeof(double) * (size_t)(NB > 0 ? NB : 1));
  double *divc = (double *)malloc(sizeof(double) * (size_t)N);
  int rc = 0;
  if (!diag || !upper || !source || !T_old || !G || !Tb || !divc) rc = -1;
  for (int32_t s = 0; s < n_steps && rc == 0; ++s) {
    memcpy(T_old, T, sizeof(double) * (size_t)N);
    ora_stats total;
    memset(&total, 0, sizeof(total));
    for (int32_t pass = 0; pass <= n_corr && rc == 0; ++pass) {
      ora_boundary_values(NB, bcell, btype, bvalue, T, Tb);
      rc = ora_gauss_grad(N, F, NB, owner, neighbour, Sf, w, V, bcell, bSf, Tb, T, G);
      if (rc) break;
      ora_assemble(N, F, owner, neighbour, V, magSf, nonOrthDelta, DTf, NB, bcell, btype, bvalue, bmagSf,
                   bdelta, DTb, dt, T_old, Su, Sp, diag, upper, source);
      /* explicit correction flux, surface-integrated (scatter over faces), / V then * V */
      for (int64_t c = 0; c < N; ++c) divc[c] = 0.0;
      for (int64_t f = 0; f < F; ++f) {
        const double *gP = G + 3 * owner[f], *gN = G + 3 * neighbour[f], *k = corr + 3 * f;
        double gf[3];
        for (int d = 0; d < 3; ++d) gf[d] = w[f] * (gP[d] - gN[d]) + gN[d];
        double flux = DTf[f] * magSf[f] * v_dot(k, gf);
        divc[owner[f]] += flux;
        divc[neighbour[f]] -= flux;
      }
      for (int64_t c = 0; c < N; ++c) source[c] += V[c] * (divc[c] / V[c]);
      ora_stats st;
      rc = ora_pcg(N, F, owner, neighbour, diag, upper, source, T, tol, rel_tol, max_iter, min_iter, &st, NULL, 0);
      if (pass == 0) {
        total.init_res = st.init_res;
        total.norm_factor = st.norm_factor;
      }
      total.iters += st.iters;
      total.final_res = st.final_res;
      total.converged = st.converged;
      total.singular |= st.singular;
      total.nonfinite |= st.nonfinite;
    }
    stats[s] = total;
  }
  free(diag); free(upper); free(source); free(T_old); free(G); free(Tb); free(divc);
  return rc;
}

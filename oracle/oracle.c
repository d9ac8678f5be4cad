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
 * invariance, finite termination of CG, a hand-computed two-cell normFactor).
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

void ora_assemble(int64_t N, int64_t F, const int32_t *owner, const int32_t *neighbour,
                  const double *V, const double *magSf, const double *delta, const double *DTf,
                  int64_t NB, const int32_t *bcell, const int32_t *btype, const double *bvalue,
                  const double *bmagSf, const double *bdelta, const double *DTb, double dt,
                  const double *T_old, double *diag, double *upper, double *source) {
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
                double *T, ora_stats *stats) {
  double *diag = (double *)malloc(sizeof(double) * (size_t)N);
  double *upper = (double *)malloc(sizeof(double) * (size_t)(F > 0 ? F : 1));
  double *source = (double *)malloc(sizeof(double) * (size_t)N);
  double *T_old = (double *)malloc(sizeof(double) * (size_t)N);
  int rc = 0;
  if (!diag || !upper || !source || !T_old) rc = -1;
  for (int32_t s = 0; s < n_steps && rc == 0; ++s) {
    memcpy(T_old, T, sizeof(double) * (size_t)N);
    ora_assemble(N, F, owner, neighbour, V, magSf, delta, DTf, NB, bcell, btype, bvalue, bmagSf,
                 bdelta, DTb, dt, T_old, diag, upper, source);
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

// Host side of the C ABI declared in include/lapfoam.h: mesh validation, the face-to-cell
// addressing, workspace layout, uploads and the advance calls.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "lfm_internal.h"

using namespace lfm;

namespace {

thread_local std::string g_last_error;

int fail_free(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Byte layout of a case's workspace. Offsets are relative to the workspace base.
struct Layout {
  size_t sync, partials, stats;
  size_t slot_other, slot_face, face_slots, b_start, b_face, bcell, btype;
  size_t V, magSf, delta, DT, bmagSf, bdelta, bDT, bval;
  size_t diag, upper, slot_coef, src, rD, vdt, x, x_old, vSu, vSp, r, w, p, q, Tb;
  size_t Sf, fw, corr, bSf, gE, gD, gH, cK, cL, grad;  // general geometry (0 when absent)
  size_t diag32, slot_coef32, rD32, dx32, r32, w32, p32, q32;
  size_t x2, xlo, xolo, e2, diag2, rD2, vdt2, g2;  // df64 form (0 when absent)
  size_t gE2, cK2, cL2, gZ, grad2;                  // df64 form on general geometry
  size_t flags;
  size_t total;
};

// kind: LFM_FP64 (FP64 solver vectors), LFM_MIXED (FP32 matrix copy + FP32 vectors, plus the
// df64 block for its outer passes), LFM_DF64 (the FP64 solver vectors, used as double-float
// pairs by the df64 form, plus the df64 block: field, diagonal, reciprocal, V/dt and slot
// conductances) or kLayoutBoth (every set, so that the precision may change after upload).
constexpr int kLayoutBoth = -1;

int layout_kind(int32_t precision) {
  return (precision == LFM_FP64 || precision == LFM_MIXED || precision == LFM_DF64) ? precision : kLayoutBoth;
}
bool kind_has64(int kind) { return kind != LFM_MIXED; }
bool kind_has32(int kind) { return kind == LFM_MIXED || kind == kLayoutBoth; }
bool kind_hasdf(int kind) { return kind != LFM_FP64; }  // the df64 form and the mixed form's outer passes

// shared_mesh: the mesh arrays (slots, boundary lists, geometry) live in another context.
// geom: general (non-orthogonal) geometry arrays and the per-case gradient / correction flux.
Layout make_layout(int64_t N, int64_t F, int64_t NB, int64_t W, int kind, bool shared_mesh = false,
                   bool geom = false) {
  Layout L{};
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = align_up(o + (bytes ? bytes : 1), 256);
    return at;
  };
  L.sync = take(sizeof(SyncWords));
  L.partials = take(sizeof(double) * kMaxCtas * kMaxSums);
  L.stats = take(sizeof(lfm_step_stats) * kStatsCap);
  L.flags = take(256);
  if (!shared_mesh) {
    L.slot_other = take(4 * W * N);
    L.slot_face = take(4 * W * N);
    L.face_slots = take(8 * F);
    L.b_start = take(4 * (N + 1));
    L.b_face = take(4 * NB);
    L.bcell = take(4 * NB);
    L.V = take(8 * N);
    L.magSf = take(8 * F);
    L.delta = take(8 * F);
    L.bmagSf = take(8 * NB);
    L.bdelta = take(8 * NB);
    if (geom) {
      L.Sf = take(24 * F);
      L.fw = take(8 * F);
      L.corr = take(24 * F);
      L.bSf = take(24 * NB);
      L.gE = take(24 * W * N);
    }
  }
  if (geom) {
    L.grad = take(24 * N);
    L.gD = take(24 * N);
    L.gH = take(24 * N);
    L.cK = take(24 * N);
    L.cL = take(24 * W * N);
  }
  L.btype = take(4 * NB);
  L.DT = take(8 * F);
  L.bDT = take(8 * NB);
  L.bval = take(8 * NB);
  L.diag = take(8 * N);
  L.upper = take(8 * F);
  L.slot_coef = take(8 * W * N);
  L.src = take(8 * N);
  L.rD = take(8 * N);
  L.vdt = take(8 * N);
  L.x = take(8 * N);
  L.x_old = take(8 * N);
  L.vSu = take(8 * N);
  L.vSp = take(8 * N);
  L.Tb = take(8 * NB);
  L.r = L.w = L.p = L.q = 0;
  L.diag32 = L.slot_coef32 = L.rD32 = L.dx32 = L.r32 = L.w32 = L.p32 = L.q32 = 0;
  L.x2 = L.xlo = L.xolo = L.e2 = L.diag2 = L.rD2 = L.vdt2 = L.g2 = 0;
  L.gE2 = L.cK2 = L.cL2 = L.gZ = L.grad2 = 0;
  if (kind_has64(kind)) {
    L.r = take(8 * N);
    L.w = take(8 * N);
    L.p = take(8 * N);
    L.q = take(8 * N);
  }
  if (kind_hasdf(kind)) {
    L.x2 = take(8 * N);
    L.xlo = take(4 * N);
    L.xolo = take(4 * N);
    L.e2 = take(8 * N);
    L.diag2 = take(8 * N);
    L.rD2 = take(8 * N);
    L.vdt2 = take(8 * N);
    L.g2 = take(8 * W * N);
    if (geom && kind != LFM_MIXED) {  // the mixed form keeps FP64 outer passes on general meshes
      L.gE2 = take(24 * W * N);
      L.cK2 = take(24 * N);
      L.cL2 = take(24 * W * N);
      L.gZ = take(24 * N);
      L.grad2 = take(24 * N);
    }
  }
  if (kind_has32(kind)) {
    L.diag32 = take(4 * N);
    L.slot_coef32 = take(4 * W * N);
    L.rD32 = take(4 * N);
    L.dx32 = take(4 * N);
    L.r32 = take(4 * N);
    L.w32 = take(4 * N);
    L.p32 = take(4 * N);
    L.q32 = take(4 * N);
  }
  L.total = o;
  return L;
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

}  // namespace

int lfm::set_last_error(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

struct lfm_batch;

struct lfm_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;

  // workspace
  char* ws = nullptr;
  size_t ws_bytes = 0;
  bool ws_owned = false;
  bool ws_bound = false;
  int ws_kind = -1;                   // solver buffers a bound workspace holds

  // case
  bool uploaded = false;
  int32_t N = 0, F = 0, NB = 0, W = 0;
  int32_t n_patches = 0;
  std::vector<int32_t> patch_start, patch_size, patch_type;
  Layout lay{};
  CaseDev cs{};

  // controls
  double dt = 1.0;
  lfm_solver_opts opts{1e-6, 0.0, 1000, 0, LFM_FP64};
  bool has64 = false, has32 = false;  // solver blocks present in the workspace
  bool hasdf = false;                 // df64 block present
  bool df_dirty = true;               // df64 conductances / V/dt to rebuild before the next df64 launch
  bool coef_dirty = true;             // FP64 / FP32 slot coefficients to rebuild before the next launch
  double mean_V = 1.0;                // mean cell volume (sets the df64 scale with dt)
  bool has_geom = false;              // general geometry uploaded (corrected laplacian)
  bool ops_dirty = false;             // operator weights to rebuild before the next launch
  bool has_Su = false, has_Sp = false;  // volumetric source set (lfm_set_source)
  int32_t n_corr = 0;                 // non-orthogonal corrector passes per step

  // launch
  int tuned_ctas = 1, tuned_threads = 512;
  int ctas = 0, threads = 0;  // overrides (0 = tuned)
  uint64_t timeout_ns = 2000000000ull;
  int skip_cta = -1;
  int stage_rows = 1;  // bulk-staged matrix rows where a pass supports them
  int skip_copy_cta = -1;

  // async state
  lfm_step_stats* h_stats = nullptr;  // pinned, kStatsCap records
  int32_t* h_status = nullptr;        // pinned
  unsigned long long* h_phase = nullptr;  // pinned, kPhases + 1 (the phase times, then the staged-pass count)
  long long staged_passes = 0;        // passes of the last advance with staged rows (team rank 0)
  double phase_ms[kPhases] = {};      // per phase kind, summed over the last advance
  cudaEvent_t done = nullptr;
  int pending_steps = 0;
  int pending_remaining = 0;
  std::vector<lfm_step_stats> stats_acc;
  lfm_batch* batch = nullptr;         // batch this context belongs to, if any
  lfm_ctx* mesh_src = nullptr;        // context whose mesh arrays this one uses
  int n_sharers = 0;                  // contexts using this one's mesh arrays
};

namespace {

int fail(lfm_ctx* c, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  g_last_error = buf;
  return code;
}

int cuda_fail(lfm_ctx* c, cudaError_t e, const char* what) {
  return fail(c, LFM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(ctx, call)                                        \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

int set_why(std::string& why, const char* fmt, ...) {
  char buf[256];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  why = buf;
  return LFM_EINVAL;
}

int check_mesh(const lfm_mesh* m, std::string& why) {
  if (!m) return set_why(why, "mesh is NULL");
  if (m->n_cells <= 0) return set_why(why, "n_cells must be > 0 (got %d)", m->n_cells);
  if (m->n_faces < 0 || m->n_bfaces < 0 || m->n_patches < 0)
    return set_why(why, "negative face or patch count (%d, %d, %d)", m->n_faces, m->n_bfaces, m->n_patches);
  if (m->n_faces > 0 && (!m->owner || !m->neighbour || !m->magSf || !m->deltaCoeffs))
    return set_why(why, "internal-face arrays missing");
  if (!m->V) return set_why(why, "V missing");
  if (m->n_bfaces > 0 && (!m->bface_cell || !m->bmagSf || !m->bdeltaCoeffs))
    return set_why(why, "boundary-face arrays missing");
  if (m->n_patches > 0 && (!m->patch_start || !m->patch_size)) return set_why(why, "patch arrays missing");
  const int64_t N = m->n_cells;
  for (int64_t c = 0; c < N; ++c)
    if (!(std::isfinite(m->V[c]) && m->V[c] > 0)) return set_why(why, "V[%lld] not finite and > 0", (long long)c);
  for (int64_t f = 0; f < m->n_faces; ++f) {
    int32_t o = m->owner[f], n = m->neighbour[f];
    if (o < 0 || o >= N || n < 0 || n >= N) return set_why(why, "face %lld: cell index out of range", (long long)f);
    if (o >= n) return set_why(why, "face %lld: owner %d >= neighbour %d", (long long)f, o, n);
    if (f > 0) {
      int32_t po = m->owner[f - 1], pn = m->neighbour[f - 1];
      if (po > o || (po == o && pn >= n)) return set_why(why, "face %lld breaks upper-triangular order", (long long)f);
    }
    if (!(std::isfinite(m->magSf[f]) && m->magSf[f] > 0)) return set_why(why, "magSf[%lld] not finite and > 0", (long long)f);
    if (!(std::isfinite(m->deltaCoeffs[f]) && m->deltaCoeffs[f] > 0))
      return set_why(why, "deltaCoeffs[%lld] not finite and > 0", (long long)f);
  }
  for (int64_t b = 0; b < m->n_bfaces; ++b) {
    int32_t c = m->bface_cell[b];
    if (c < 0 || c >= N) return set_why(why, "boundary face %lld: cell %d out of range", (long long)b, c);
    if (!(std::isfinite(m->bmagSf[b]) && m->bmagSf[b] > 0)) return set_why(why, "bmagSf[%lld] not finite and > 0", (long long)b);
    if (!(std::isfinite(m->bdeltaCoeffs[b]) && m->bdeltaCoeffs[b] > 0))
      return set_why(why, "bdeltaCoeffs[%lld] not finite and > 0", (long long)b);
  }
  int64_t at = 0;
  for (int32_t p = 0; p < m->n_patches; ++p) {
    if (m->patch_start[p] != at || m->patch_size[p] < 0)
      return set_why(why, "patch %d does not continue the boundary faces at %lld", p, (long long)at);
    at += m->patch_size[p];
  }
  if (at != m->n_bfaces) return set_why(why, "patches cover %lld of %d boundary faces", (long long)at, m->n_bfaces);
  return LFM_OK;
}

// Geometry of a general mesh: finite values, weights in [0, 1], |Sf| consistent with magSf.
int check_geometry(const lfm_mesh* m, const lfm_geometry* g, std::string& why) {
  if ((m->n_faces > 0 && (!g->Sf || !g->weights || !g->corr_vec)) || (m->n_bfaces > 0 && !g->bSf))
    return set_why(why, "geometry arrays missing");
  for (int64_t f = 0; f < m->n_faces; ++f) {
    const double* s = g->Sf + 3 * f;
    const double* k = g->corr_vec + 3 * f;
    const double w = g->weights[f];
    if (!(std::isfinite(w) && w >= 0.0 && w <= 1.0)) return set_why(why, "weights[%lld] not in [0, 1]", (long long)f);
    for (int d = 0; d < 3; ++d)
      if (!std::isfinite(s[d]) || !std::isfinite(k[d])) return set_why(why, "face %lld: Sf or corr_vec not finite", (long long)f);
    const double mag = std::sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
    if (!(std::fabs(mag - m->magSf[f]) <= 1e-9 * m->magSf[f]))
      return set_why(why, "face %lld: |Sf| = %g differs from magSf = %g", (long long)f, mag, m->magSf[f]);
  }
  for (int64_t b = 0; b < m->n_bfaces; ++b) {
    const double* s = g->bSf + 3 * b;
    for (int d = 0; d < 3; ++d)
      if (!std::isfinite(s[d])) return set_why(why, "boundary face %lld: bSf not finite", (long long)b);
    const double mag = std::sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
    if (!(std::fabs(mag - m->bmagSf[b]) <= 1e-9 * m->bmagSf[b]))
      return set_why(why, "boundary face %lld: |bSf| differs from bmagSf", (long long)b);
  }
  return LFM_OK;
}

// Counting sort by key (stable): start[k] .. start[k+1] index the items with key k, in
// ascending item order.
void bucket(int32_t n_keys, int64_t n_items, const int32_t* key, int32_t* start, int32_t* order) {
  std::fill(start, start + n_keys + 1, 0);
  for (int64_t i = 0; i < n_items; ++i) ++start[key[i] + 1];
  for (int32_t k = 0; k < n_keys; ++k) start[k + 1] += start[k];
  std::vector<int32_t> fill(start, start + n_keys);
  for (int64_t i = 0; i < n_items; ++i) order[fill[key[i]]++] = (int32_t)i;
}

// Largest number of internal faces of any cell (the slot width of the layout).
int32_t slot_width(const lfm_mesh* m) {
  std::vector<int32_t> deg(m->n_cells, 0);
  for (int32_t f = 0; f < m->n_faces; ++f) {
    ++deg[m->owner[f]];
    ++deg[m->neighbour[f]];
  }
  int32_t W = 0;
  for (int32_t v : deg) W = v > W ? v : W;
  return W;
}

template <class T>
int h2d(lfm_ctx* c, size_t off, const T* src, size_t n) {
  if (n == 0) return LFM_OK;
  CK(c, cudaMemcpyAsync(c->ws + off, src, sizeof(T) * n, cudaMemcpyHostToDevice, c->stream));
  return LFM_OK;
}

// Default launch: one team of co-resident CTAs of 512 threads, at least about 4096 cells
// per CTA (the best shape in launch-shape sweeps on the 200^3 graded box).
int choose_launch(lfm_ctx* c) {
  const int threads = 512;
  int maxc = max_coresident_ctas(c->opts.precision, threads, c->W, c->device);
  if (maxc <= 0) return fail(c, LFM_ECUDA, "cannot size the cooperative launch");
  int64_t want = ((int64_t)c->N + 4095) / 4096;
  if (want < 1) want = 1;
  if (want > maxc) want = maxc;
  c->tuned_ctas = (int)want;
  c->tuned_threads = threads;
  return LFM_OK;
}

Launch current_launch(lfm_ctx* c, int& err) {
  Launch L{};
  L.threads = c->threads > 0 ? c->threads : c->tuned_threads;
  int maxc = max_coresident_ctas(c->opts.precision, L.threads, c->W, c->device);
  L.ctas = c->ctas > 0 ? c->ctas : c->tuned_ctas;
  if (L.ctas > maxc) L.ctas = maxc;
  err = L.ctas <= 0 ? 1 : 0;
  L.timeout_ns = c->timeout_ns;
  L.skip_cta = c->skip_cta;
  L.stage_rows = c->stage_rows;
  L.skip_copy_cta = c->skip_copy_cta;
  return L;
}

void refresh_case(lfm_ctx* c) {
  CaseDev& cs = c->cs;
  cs.dt = c->dt;
  cs.tol = c->opts.tol;
  cs.rel_tol = c->opts.rel_tol;
  cs.max_iter = c->opts.max_iter;
  cs.min_iter = c->opts.min_iter;
  cs.precision = c->opts.precision;
  cs.n_corr = c->n_corr;
}

// Power-of-two scale of the df64 form's system: V/dt near one for a cell of mean volume.
double df_scale_for(double mean_V, double dt) {
  const double v = mean_V / dt;
  if (!(std::isfinite(v) && v > 0)) return 1.0;
  long k = std::lround(std::log2(v));
  if (k > 900) k = 900;
  if (k < -900) k = -900;
  return std::ldexp(1.0, (int)-k);
}

void bind_pointers(lfm_ctx* c) {
  const Layout& L = c->lay;
  char* b = c->ws;
  CaseDev& cs = c->cs;
  cs.N = c->N;
  cs.F = c->F;
  cs.NB = c->NB;
  cs.sync = reinterpret_cast<SyncWords*>(b + L.sync);
  cs.partials = reinterpret_cast<double*>(b + L.partials);
  cs.stats = reinterpret_cast<lfm_step_stats*>(b + L.stats);
  cs.flags = reinterpret_cast<int32_t*>(b + L.flags);
  cs.seed_sums = reinterpret_cast<double*>(b + L.flags + 64);
  cs.W = c->W;
  cs.btype = reinterpret_cast<const int32_t*>(b + L.btype);
  cs.DT = reinterpret_cast<const double*>(b + L.DT);
  cs.bDT = reinterpret_cast<const double*>(b + L.bDT);
  cs.bval = reinterpret_cast<const double*>(b + L.bval);
  if (c->mesh_src) {
    const CaseDev& m = c->mesh_src->cs;
    cs.slot_other = m.slot_other;
    cs.slot_face = m.slot_face;
    cs.face_slots = m.face_slots;
    cs.b_start = m.b_start;
    cs.b_face = m.b_face;
    cs.bcell = m.bcell;
    cs.V = m.V;
    cs.magSf = m.magSf;
    cs.delta = m.delta;
    cs.bmagSf = m.bmagSf;
    cs.bdelta = m.bdelta;
    cs.Sf = m.Sf;
    cs.fw = m.fw;
    cs.corr = m.corr;
    cs.bSf = m.bSf;
    cs.gE = m.gE;
  } else {
    cs.slot_other = reinterpret_cast<const int32_t*>(b + L.slot_other);
    cs.slot_face = reinterpret_cast<const int32_t*>(b + L.slot_face);
    cs.face_slots = reinterpret_cast<const uint32_t*>(b + L.face_slots);
    cs.b_start = reinterpret_cast<const int32_t*>(b + L.b_start);
    cs.b_face = reinterpret_cast<const int32_t*>(b + L.b_face);
    cs.bcell = reinterpret_cast<const int32_t*>(b + L.bcell);
    cs.V = reinterpret_cast<const double*>(b + L.V);
    cs.magSf = reinterpret_cast<const double*>(b + L.magSf);
    cs.delta = reinterpret_cast<const double*>(b + L.delta);
    cs.bmagSf = reinterpret_cast<const double*>(b + L.bmagSf);
    cs.bdelta = reinterpret_cast<const double*>(b + L.bdelta);
    const bool g = c->has_geom;
    cs.Sf = g ? reinterpret_cast<const double*>(b + L.Sf) : nullptr;
    cs.fw = g ? reinterpret_cast<const double*>(b + L.fw) : nullptr;
    cs.corr = g ? reinterpret_cast<const double*>(b + L.corr) : nullptr;
    cs.bSf = g ? reinterpret_cast<const double*>(b + L.bSf) : nullptr;
    cs.gE = g ? reinterpret_cast<const double*>(b + L.gE) : nullptr;
  }
  const bool gc = c->has_geom;
  cs.grad = gc ? reinterpret_cast<double*>(b + L.grad) : nullptr;
  cs.gD = gc ? reinterpret_cast<const double*>(b + L.gD) : nullptr;
  cs.gH = gc ? reinterpret_cast<const double*>(b + L.gH) : nullptr;
  cs.cK = gc ? reinterpret_cast<const double*>(b + L.cK) : nullptr;
  cs.cL = gc ? reinterpret_cast<const double*>(b + L.cL) : nullptr;
  cs.x_old = reinterpret_cast<double*>(b + L.x_old);
  cs.vSu = c->has_Su ? reinterpret_cast<const double*>(b + L.vSu) : nullptr;
  cs.vSp = c->has_Sp ? reinterpret_cast<const double*>(b + L.vSp) : nullptr;
  cs.diag = reinterpret_cast<double*>(b + L.diag);
  cs.upper = reinterpret_cast<double*>(b + L.upper);
  cs.slot_coef = reinterpret_cast<double*>(b + L.slot_coef);
  cs.src = reinterpret_cast<double*>(b + L.src);
  cs.rD = reinterpret_cast<double*>(b + L.rD);
  cs.vdt = reinterpret_cast<const double*>(b + L.vdt);
  cs.x = reinterpret_cast<double*>(b + L.x);
  const bool d = c->has64, m = c->has32;
  cs.r = d ? reinterpret_cast<double*>(b + L.r) : nullptr;
  cs.w = d ? reinterpret_cast<double*>(b + L.w) : nullptr;
  cs.p = d ? reinterpret_cast<double*>(b + L.p) : nullptr;
  cs.q = d ? reinterpret_cast<double*>(b + L.q) : nullptr;
  cs.diag32 = m ? reinterpret_cast<float*>(b + L.diag32) : nullptr;
  cs.slot_coef32 = m ? reinterpret_cast<float*>(b + L.slot_coef32) : nullptr;
  cs.rD32 = m ? reinterpret_cast<float*>(b + L.rD32) : nullptr;
  cs.dx32 = m ? reinterpret_cast<float*>(b + L.dx32) : nullptr;
  cs.r32 = m ? reinterpret_cast<float*>(b + L.r32) : nullptr;
  cs.w32 = m ? reinterpret_cast<float*>(b + L.w32) : nullptr;
  cs.p32 = m ? reinterpret_cast<float*>(b + L.p32) : nullptr;
  cs.q32 = m ? reinterpret_cast<float*>(b + L.q32) : nullptr;
  const bool f = c->hasdf;
  cs.x2 = f ? reinterpret_cast<float2*>(b + L.x2) : nullptr;
  cs.xlo = f ? reinterpret_cast<float*>(b + L.xlo) : nullptr;
  cs.xolo = f ? reinterpret_cast<float*>(b + L.xolo) : nullptr;
  cs.e2 = f ? reinterpret_cast<float2*>(b + L.e2) : nullptr;
  const bool fg = f && c->has_geom && L.gE2 != 0;
  cs.gE2 = fg ? reinterpret_cast<const float2*>(b + L.gE2) : nullptr;
  cs.cK2 = fg ? reinterpret_cast<const float2*>(b + L.cK2) : nullptr;
  cs.cL2 = fg ? reinterpret_cast<const float2*>(b + L.cL2) : nullptr;
  cs.gZ = fg ? reinterpret_cast<const float2*>(b + L.gZ) : nullptr;
  cs.grad2 = fg ? reinterpret_cast<float2*>(b + L.grad2) : nullptr;
  cs.diag2 = f ? reinterpret_cast<float2*>(b + L.diag2) : nullptr;
  cs.rD2 = f ? reinterpret_cast<float2*>(b + L.rD2) : nullptr;
  cs.vdt2 = f ? reinterpret_cast<const float2*>(b + L.vdt2) : nullptr;
  cs.g2 = f ? reinterpret_cast<const float2*>(b + L.g2) : nullptr;
  cs.df_scale = df_scale_for(c->mean_V, c->dt);
}

// V/dt per cell, recomputed when dt or the mesh changes (the assembly reads it every step).
bool ctx_batch_pending(const lfm_ctx* c);

int refresh_vdt(lfm_ctx* c) {
  CK(c, launch_vdt(c->cs.V, c->dt, const_cast<double*>(c->cs.vdt), c->N, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  c->cs.df_scale = df_scale_for(c->mean_V, c->dt);
  c->df_dirty = true;
  return LFM_OK;
}

// Rebuilds the face coefficients of the slot arrays (a0) when the mesh or DT changed since
// they were built (the df64 form keeps its own, see refresh_df).
int refresh_coef(lfm_ctx* c) {
  if (!c->coef_dirty || c->opts.precision == LFM_DF64) return LFM_OK;
  CK(c, launch_coef_setup(c->cs, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  c->coef_dirty = false;
  return LFM_OK;
}

// Rebuilds the df64 conductances and V/dt (a0 of the df64 form) when the mesh, DT or dt
// changed since they were built. Enqueued on the context's stream.
int refresh_df(lfm_ctx* c) {
  const bool want = c->opts.precision == LFM_DF64 || (c->opts.precision == LFM_MIXED && c->hasdf && !c->has_geom);
  if (!want || !c->df_dirty) return LFM_OK;
  if (!c->hasdf) return fail(c, LFM_ENOMEM, "the workspace has no df64 buffers");
  CK(c, launch_df_setup(c->cs, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));  // batches launch on their own stream
  c->df_dirty = false;
  return LFM_OK;
}

// Rebuilds the case's operator weights (general geometry) when patches, boundary values or
// DT changed since the last launch. Enqueued on the context's stream.
int refresh_ops(lfm_ctx* c) {
  if (!c->has_geom || !c->ops_dirty) return LFM_OK;
  refresh_case(c);
  CK(c, launch_geom_ops(c->cs, false, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));  // batches launch on their own stream
  c->ops_dirty = false;
  c->df_dirty = true;  // the df64 copies of the operators follow them
  return LFM_OK;
}

// The FP64 field is about to be written other than by a df64 launch: the triple-float copy
// the df64 forms carry across launches is stale from then on (see lfm_solve_df.cuh), and so
// is the mixed form's seed of its next step (flags[1]).
int invalidate_split(lfm_ctx* c) {
  CK(c, cudaMemsetAsync(c->cs.flags, 0, 2 * sizeof(int32_t), c->stream));
  return LFM_OK;
}

// The case changed (its matrix, source, controls or launch shape): the next step's rows and
// inner-solve seed that the mixed form's last launch left in place no longer apply
// (lfm_solve_mixed_df.cuh). Stream-ordered after any launch still pending.
int invalidate_seed(lfm_ctx* c) {
  DeviceGuard g(c->device);
  CK(c, cudaMemsetAsync(c->cs.flags + 1, 0, sizeof(int32_t), c->stream));
  return LFM_OK;
}

int need_uploaded(lfm_ctx* c) {
  if (!c) return fail_free(LFM_EINVAL, "context is NULL");
  if (!c->uploaded) return fail(c, LFM_ESTATE, "no mesh uploaded");
  return LFM_OK;
}

// Enqueues one launch of `steps` steps (<= kStatsCap) and the copy-back of its statistics
// and status into pinned host memory.
int enqueue_chunk(lfm_ctx* c, int steps, int mode) {
  refresh_case(c);
  if (int rc = refresh_ops(c)) return rc;
  if (mode == kModeSteps) {
    if (int rc = refresh_coef(c)) return rc;
    if (int rc = refresh_df(c)) return rc;
    const int p = c->opts.precision;
    if (p == LFM_FP64 || (p == LFM_MIXED && !mixed_runs_df(c->cs))) {
      if (int rc = invalidate_split(c)) return rc;
    } else if (p == LFM_DF64) {
      if (int rc = invalidate_seed(c)) return rc;
    }
  }
  int e = 0;
  Launch L = current_launch(c, e);
  if (e) return fail(c, LFM_ECUDA, "no co-resident CTA fits the step kernel");
  if (mode == kModeAssembleOnly && c->opts.precision == LFM_DF64) {  // read-back runs the FP64 assembly
    const int m = max_coresident_ctas(LFM_FP64, L.threads, c->W, c->device);
    if (L.ctas > m) L.ctas = m;
    if (L.ctas <= 0) return fail(c, LFM_ECUDA, "no co-resident CTA fits the assembly kernel");
  }
  if (L.skip_cta >= 0 && L.ctas < 2) return fail(c, LFM_EINVAL, "the skip-arrival hook needs >= 2 CTAs");
  CK(c, cudaMemsetAsync(c->cs.sync, 0, sizeof(SyncWords), c->stream));
  CK(c, launch_steps(c->cs, L, steps, mode, c->stream));
  c->skip_cta = -1;
  c->skip_copy_cta = -1;
  if (steps > 0)
    CK(c, cudaMemcpyAsync(c->h_stats, c->cs.stats, sizeof(lfm_step_stats) * steps, cudaMemcpyDeviceToHost,
                          c->stream));
  CK(c, cudaMemcpyAsync(c->h_status, &c->cs.sync->status, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaMemcpyAsync(c->h_phase, c->cs.sync->phase_ns, sizeof(unsigned long long) * (kPhases + 1),
                        cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaEventRecord(c->done, c->stream));
  return LFM_OK;
}

// Checked build: the first index check that failed in a kernel since the last take.
int take_checks(lfm_ctx* c) {
  if (!kCheckedBuild) return LFM_OK;
  int site = check_take_step(c->stream);
  if (site == 0) site = check_take_batch(c->stream);
  if (site < 0) return fail(c, LFM_ECUDA, "reading the index-check word failed");
  if (site > 0) return fail(c, LFM_EINVAL, "checked build: a kernel met an index out of range (check site %d)", site);
  return LFM_OK;
}

// Waits for the enqueued chunk, appends its statistics, maps the device status.
int collect_chunk(lfm_ctx* c, int steps) {
  CK(c, cudaEventSynchronize(c->done));
  for (int i = 0; i < steps; ++i) c->stats_acc.push_back(c->h_stats[i]);
  for (int k = 0; k < kPhases; ++k) c->phase_ms[k] += 1e-6 * (double)c->h_phase[k];
  c->staged_passes += (long long)c->h_phase[kPhases];
  int32_t st = *c->h_status;
  if (st != 0) invalidate_seed(c);  // a launch that stopped early left no seed to trust
  if (st == LFM_ETIMEOUT) return fail(c, LFM_ETIMEOUT, "a device barrier wait ran out (kernel stopped)");
  if (st == LFM_ESINGULAR) return fail(c, LFM_ESINGULAR, "PCG met a singular search direction");
  if (st == LFM_ENONFINITE) return fail(c, LFM_ENONFINITE, "PCG residual became non-finite");
  if (st != 0) return fail(c, LFM_ECUDA, "device status %d", (int)st);
  return take_checks(c);
}

}  // namespace

extern "C" {

const char* lfm_version(void) { return "lapfoam-gb300 0.1 (sm_103a)"; }

int lfm_mesh_check(const lfm_mesh* mesh, char* msg, size_t msg_len) {
  std::string why;
  int rc = check_mesh(mesh, why);
  if (msg && msg_len) {
    snprintf(msg, msg_len, "%s", rc == LFM_OK ? "" : why.c_str());
  }
  if (rc != LFM_OK) g_last_error = why;
  return rc;
}

int lfm_face_addressing(int32_t n_cells, int32_t n_faces, const int32_t* owner, const int32_t* neighbour,
                        int32_t* own_start, int32_t* losort, int32_t* lo_start) {
  if (n_cells <= 0 || n_faces < 0 || (n_faces > 0 && (!owner || !neighbour)) || !own_start || !lo_start ||
      (n_faces > 0 && !losort))
    return fail_free(LFM_EINVAL, "lfm_face_addressing: bad arguments");
  for (int32_t f = 0; f < n_faces; ++f) {
    if (owner[f] < 0 || owner[f] >= n_cells || neighbour[f] <= owner[f] || neighbour[f] >= n_cells)
      return fail_free(LFM_EINVAL, "lfm_face_addressing: face %d out of range or owner >= neighbour", f);
    if (f > 0 && owner[f] < owner[f - 1])
      return fail_free(LFM_EINVAL, "lfm_face_addressing: faces not sorted by owner at %d", f);
  }
  std::vector<int32_t> order(n_faces > 0 ? n_faces : 1);
  bucket(n_cells, n_faces, owner, own_start, order.data());  // identity order: faces sorted by owner
  bucket(n_cells, n_faces, neighbour, lo_start, losort);
  return LFM_OK;
}

size_t lfm_workspace_bytes(const lfm_mesh* mesh, int32_t precision) {
  std::string why;
  if (check_mesh(mesh, why) != LFM_OK) {
    g_last_error = why;
    return 0;
  }
  precision = layout_kind(precision);
  return make_layout(mesh->n_cells, mesh->n_faces, mesh->n_bfaces, slot_width(mesh), precision).total;
}

int lfm_create(lfm_ctx** out, int device, void* cuda_stream) {
  if (!out) return fail_free(LFM_EINVAL, "lfm_create: out is NULL");
  *out = nullptr;
  int n = 0;
  cudaError_t e = cudaGetDeviceCount(&n);
  if (e != cudaSuccess || n == 0) return fail_free(LFM_ECUDA, "no CUDA device (%s)", cudaGetErrorString(e));
  if (device < 0 || device >= n) return fail_free(LFM_EINVAL, "device %d out of range", device);
  lfm_ctx* c = new (std::nothrow) lfm_ctx;
  if (!c) return fail_free(LFM_ENOMEM, "out of host memory");
  c->device = device;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  DeviceGuard g(device);
  if (cudaMallocHost(&c->h_stats, sizeof(lfm_step_stats) * kStatsCap) != cudaSuccess ||
      cudaMallocHost(&c->h_status, sizeof(int32_t)) != cudaSuccess ||
      cudaMallocHost(&c->h_phase, sizeof(unsigned long long) * (kPhases + 1)) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->done, cudaEventDisableTiming) != cudaSuccess) {
    lfm_destroy(c);
    return fail_free(LFM_ECUDA, "lfm_create: host staging or event allocation failed");
  }
  *out = c;
  return LFM_OK;
}

int lfm_bind_workspace(lfm_ctx* c, void* dev_ptr, size_t bytes, int32_t precision) {
  if (!c) return fail_free(LFM_EINVAL, "context is NULL");
  if (c->uploaded) return fail(c, LFM_ESTATE, "bind the workspace before uploading a mesh");
  if (!dev_ptr || (reinterpret_cast<uintptr_t>(dev_ptr) & 255)) return fail(c, LFM_EINVAL, "workspace must be 256-byte aligned");
  c->ws = static_cast<char*>(dev_ptr);
  c->ws_bytes = bytes;
  c->ws_bound = true;
  c->ws_owned = false;
  c->ws_kind = layout_kind(precision);
  return LFM_OK;
}

static int upload_mesh_impl(lfm_ctx* c, const lfm_mesh* m, const lfm_geometry* geo) {
  if (!c) return fail_free(LFM_EINVAL, "context is NULL");
  if (c->n_sharers > 0 || c->mesh_src) return fail(c, LFM_ESTATE, "the context shares a mesh");
  std::string why;
  if (check_mesh(m, why) != LFM_OK) return fail(c, LFM_EINVAL, "%s", why.c_str());
  if (geo && check_geometry(m, geo, why) != LFM_OK) return fail(c, LFM_EINVAL, "%s", why.c_str());
  DeviceGuard g(c->device);
  const int32_t W = slot_width(m);
  if (W > kMaxSlots) return fail(c, LFM_EINVAL, "a cell has %d internal faces (at most %d supported)", W, kMaxSlots);
  if ((uint64_t)W * (uint64_t)m->n_cells > 0xffffffffull)
    return fail(c, LFM_EINVAL, "slot width x cells = %llu exceeds 2^32 - 1",
                (unsigned long long)W * (unsigned long long)m->n_cells);
  const int kind = c->ws_bound ? c->ws_kind : kLayoutBoth;
  const Layout use = make_layout(m->n_cells, m->n_faces, m->n_bfaces, W, kind, false, geo != nullptr);
  const bool has64 = kind_has64(kind), has32 = kind_has32(kind), hasdf = kind_hasdf(kind);
  if (c->ws_bound) {
    if (c->ws_bytes < use.total) return fail(c, LFM_ENOMEM, "workspace has %zu bytes, needs %zu", c->ws_bytes, use.total);
  } else {
    if (c->ws_owned && c->ws) {
      cudaFree(c->ws);
      c->ws = nullptr;
    }
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, use.total);
    if (e != cudaSuccess) return fail(c, LFM_ENOMEM, "device allocation of %zu bytes failed: %s", use.total, cudaGetErrorString(e));
    c->ws = static_cast<char*>(p);
    c->ws_bytes = use.total;
    c->ws_owned = true;
  }
  c->lay = use;
  {
    double sv = 0.0;
    for (int32_t i = 0; i < m->n_cells; ++i) sv += m->V[i];
    c->mean_V = sv / (double)m->n_cells;
  }
  c->N = m->n_cells;
  c->F = m->n_faces;
  c->NB = m->n_bfaces;
  c->W = W;
  c->has64 = has64;
  c->has32 = has32;
  c->hasdf = hasdf;
  c->df_dirty = true;
  c->coef_dirty = true;
  c->has_geom = geo != nullptr;
  c->n_corr = 0;
  c->has_Su = c->has_Sp = false;
  c->n_patches = m->n_patches;
  c->patch_start.assign(m->patch_start, m->patch_start + m->n_patches);
  c->patch_size.assign(m->patch_size, m->patch_size + m->n_patches);
  c->patch_type.assign(m->n_patches, LFM_ZERO_GRADIENT);
  bind_pointers(c);
  if (int e = invalidate_split(c)) return e;

  const int32_t N = c->N, F = c->F, NB = c->NB;
  int rc;
  std::vector<int32_t> btype(NB > 0 ? NB : 1, LFM_ZERO_GRADIENT);
  std::vector<double> zeros_b(NB > 0 ? NB : 1, 0.0);

  // Face-to-cell addressing and the slot-major rows, built on the device from owner,
  // neighbour and bface_cell (staged in a temporary buffer; bface_cell lands in bcell).
  const Layout& Y = c->lay;
  const size_t WN = (size_t)W * N;
  if ((rc = h2d(c, Y.bcell, m->bface_cell, NB))) return rc;
  {
    int32_t* on = nullptr;
    CK(c, cudaMalloc(&on, sizeof(int32_t) * 2 * (size_t)(F > 0 ? F : 1)));
    cudaError_t e = cudaSuccess;
    if (F > 0) {
      e = cudaMemcpyAsync(on, m->owner, sizeof(int32_t) * F, cudaMemcpyHostToDevice, c->stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(on + F, m->neighbour, sizeof(int32_t) * F, cudaMemcpyHostToDevice, c->stream);
    }
    if (e == cudaSuccess)
      e = build_addressing(N, F, NB, W, on, on + F, c->cs.bcell, const_cast<int32_t*>(c->cs.slot_other),
                           const_cast<int32_t*>(c->cs.slot_face), const_cast<uint32_t*>(c->cs.face_slots),
                           const_cast<int32_t*>(c->cs.b_start), const_cast<int32_t*>(c->cs.b_face), c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(on);
    if (e != cudaSuccess) return cuda_fail(c, e, "device face addressing");
  }
  if ((rc = h2d(c, Y.btype, btype.data(), NB)) || (rc = h2d(c, Y.V, m->V, N)) ||
      (rc = h2d(c, Y.magSf, m->magSf, F)) || (rc = h2d(c, Y.delta, m->deltaCoeffs, F)) ||
      (rc = h2d(c, Y.bmagSf, m->bmagSf, NB)) || (rc = h2d(c, Y.bdelta, m->bdeltaCoeffs, NB)) ||
      (rc = h2d(c, Y.bDT, zeros_b.data(), NB)) || (rc = h2d(c, Y.bval, zeros_b.data(), NB)))
    return rc;
  if (geo && ((rc = h2d(c, Y.Sf, geo->Sf, 3 * (size_t)F)) || (rc = h2d(c, Y.fw, geo->weights, F)) ||
              (rc = h2d(c, Y.corr, geo->corr_vec, 3 * (size_t)F)) || (rc = h2d(c, Y.bSf, geo->bSf, 3 * (size_t)NB))))
    return rc;
  c->ops_dirty = geo != nullptr;
  if (WN > 0) {
    CK(c, cudaMemsetAsync(c->ws + Y.slot_coef, 0, sizeof(double) * WN, c->stream));
    if (has32) CK(c, cudaMemsetAsync(c->ws + Y.slot_coef32, 0, sizeof(float) * WN, c->stream));
  }
  CK(c, cudaMemsetAsync(c->ws + Y.DT, 0, sizeof(double) * (F > 0 ? F : 1), c->stream));
  c->cs.DT_is_uniform = 1;
  c->cs.DT_uniform = 0.0;
  CK(c, cudaMemsetAsync(c->ws + Y.x, 0, sizeof(double) * N, c->stream));
  if (geo) {  // the geometry-only gradient weights, once per mesh (meshes sharing it read them)
    refresh_case(c);
    CK(c, launch_geom_ops(c->cs, true, c->stream));
  }
  CK(c, cudaStreamSynchronize(c->stream));
  c->dt = 1.0;
  c->opts = lfm_solver_opts{1e-6, 0.0, 1000, 0, has64 ? LFM_FP64 : LFM_MIXED};
  if ((rc = refresh_vdt(c))) return rc;
  c->uploaded = true;
  c->ctas = c->threads = 0;
  return choose_launch(c);
}

int lfm_upload_mesh(lfm_ctx* c, const lfm_mesh* m) { return upload_mesh_impl(c, m, nullptr); }

int lfm_upload_mesh_geometry(lfm_ctx* c, const lfm_mesh* m, const lfm_geometry* geometry) {
  if (!geometry) return fail(c, LFM_EINVAL, "geometry is NULL");
  return upload_mesh_impl(c, m, geometry);
}

size_t lfm_workspace_bytes_geometry(const lfm_mesh* mesh, int32_t precision) {
  std::string why;
  if (check_mesh(mesh, why) != LFM_OK) {
    g_last_error = why;
    return 0;
  }
  precision = layout_kind(precision);
  return make_layout(mesh->n_cells, mesh->n_faces, mesh->n_bfaces, slot_width(mesh), precision, false, true).total;
}

namespace {
int check_box(int32_t nx, int32_t ny, int32_t nz, const double* xs, const double* ys, const double* zs,
              std::string& why) {
  if (nx < 1 || ny < 1 || nz < 1) return set_why(why, "box dimensions must be >= 1");
  if (!xs || !ys || !zs) return set_why(why, "vertex coordinates missing");
  const long long N = (long long)nx * ny * nz;
  const long long F = (long long)(nx - 1) * ny * nz + (long long)nx * (ny - 1) * nz + (long long)nx * ny * (nz - 1);
  if (N > 0x7fffffffLL || F > 0x7fffffffLL) return set_why(why, "box too large for 32-bit indices");
  if ((long long)box_slot_width(nx, ny, nz) * N > 0xffffffffLL) return set_why(why, "slot width x cells exceeds 2^32 - 1");
  if ((long long)nx + ny + nz + 3 > (long long)kMaxCtas * kMaxSums) return set_why(why, "too many vertex planes");
  const double* ax[3] = {xs, ys, zs};
  const int32_t n[3] = {nx, ny, nz};
  for (int a = 0; a < 3; ++a)
    for (int32_t i = 0; i <= n[a]; ++i) {
      if (!std::isfinite(ax[a][i])) return set_why(why, "vertex coordinate not finite");
      if (i > 0 && !(ax[a][i] > ax[a][i - 1])) return set_why(why, "vertex coordinates must increase strictly");
    }
  return LFM_OK;
}
}  // namespace

int lfm_box_counts(int32_t nx, int32_t ny, int32_t nz, int32_t* n_cells, int32_t* n_faces, int32_t* n_bfaces,
                   int32_t* slot_width) {
  if (nx < 1 || ny < 1 || nz < 1) return fail_free(LFM_EINVAL, "box dimensions must be >= 1");
  const long long N = (long long)nx * ny * nz;
  const long long F = (long long)(nx - 1) * ny * nz + (long long)nx * (ny - 1) * nz + (long long)nx * ny * (nz - 1);
  if (N > 0x7fffffffLL || F > 0x7fffffffLL) return fail_free(LFM_EINVAL, "box too large for 32-bit indices");
  if ((long long)box_slot_width(nx, ny, nz) * N > 0xffffffffLL)
    return fail_free(LFM_EINVAL, "slot width x cells exceeds 2^32 - 1");
  if (n_cells) *n_cells = (int32_t)N;
  if (n_faces) *n_faces = (int32_t)F;
  if (n_bfaces) *n_bfaces = (int32_t)(2 * ((long long)ny * nz + (long long)nx * nz + (long long)nx * ny));
  if (slot_width) *slot_width = box_slot_width(nx, ny, nz);
  return LFM_OK;
}

int lfm_box_layout(int32_t nx, int32_t ny, int32_t nz, const double* xs, const double* ys, const double* zs,
                   int32_t* slot_other, int32_t* slot_face, uint32_t* face_slots, double* V, double* magSf,
                   double* delta,
                   int32_t* b_start, int32_t* b_face, int32_t* bcell, double* bmagSf, double* bdelta) {
  std::string why;
  if (check_box(nx, ny, nz, xs, ys, zs, why) != LFM_OK) return fail_free(LFM_EINVAL, "%s", why.c_str());
  if (!slot_other || !slot_face || !face_slots || !V || !magSf || !delta || !b_start || !b_face || !bcell ||
      !bmagSf || !bdelta)
    return fail_free(LFM_EINVAL, "output arrays missing");
  box_layout_host(nx, ny, nz, box_slot_width(nx, ny, nz), xs, ys, zs, slot_other, slot_face, face_slots, V, magSf,
                  delta,
                  b_start, b_face, bcell, bmagSf, bdelta);
  return LFM_OK;
}

int lfm_upload_box(lfm_ctx* c, int32_t nx, int32_t ny, int32_t nz, const double* xs, const double* ys,
                   const double* zs) {
  if (!c) return fail_free(LFM_EINVAL, "context is NULL");
  if (c->uploaded || c->n_sharers > 0 || c->mesh_src) return fail(c, LFM_ESTATE, "the context already has a mesh");
  std::string why;
  if (check_box(nx, ny, nz, xs, ys, zs, why) != LFM_OK) return fail(c, LFM_EINVAL, "%s", why.c_str());
  DeviceGuard g(c->device);
  int32_t N, F, NB, W;
  lfm_box_counts(nx, ny, nz, &N, &F, &NB, &W);
  const int kind = c->ws_bound ? c->ws_kind : kLayoutBoth;
  const Layout use = make_layout(N, F, NB, W, kind);
  const bool has64 = kind_has64(kind), has32 = kind_has32(kind), hasdf = kind_hasdf(kind);
  if (c->ws_bound) {
    if (c->ws_bytes < use.total) return fail(c, LFM_ENOMEM, "workspace has %zu bytes, needs %zu", c->ws_bytes, use.total);
  } else {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, use.total);
    if (e != cudaSuccess) return fail(c, LFM_ENOMEM, "device allocation of %zu bytes failed: %s", use.total, cudaGetErrorString(e));
    c->ws = static_cast<char*>(p);
    c->ws_bytes = use.total;
    c->ws_owned = true;
  }
  c->lay = use;
  c->mean_V = (xs[nx] - xs[0]) * (ys[ny] - ys[0]) * (zs[nz] - zs[0]) / (double)N;
  c->N = N;
  c->F = F;
  c->NB = NB;
  c->W = W;
  c->has64 = has64;
  c->has32 = has32;
  c->hasdf = hasdf;
  c->df_dirty = true;
  c->coef_dirty = true;
  c->has_geom = false;
  c->n_corr = 0;
  c->has_Su = c->has_Sp = false;
  c->n_patches = 6;
  const int32_t sizes[6] = {ny * nz, ny * nz, nx * nz, nx * nz, nx * ny, nx * ny};
  c->patch_start.assign(6, 0);
  c->patch_size.assign(sizes, sizes + 6);
  for (int p = 1; p < 6; ++p) c->patch_start[p] = c->patch_start[p - 1] + sizes[p - 1];
  c->patch_type.assign(6, LFM_ZERO_GRADIENT);
  bind_pointers(c);
  if (int e = invalidate_split(c)) return e;
  // vertex coordinates staged in the (not yet used) partial-sum table
  double* coords = c->cs.partials;
  const Layout& Y = c->lay;
  CK(c, cudaMemcpyAsync(coords, xs, sizeof(double) * (nx + 1), cudaMemcpyHostToDevice, c->stream));
  CK(c, cudaMemcpyAsync(coords + nx + 1, ys, sizeof(double) * (ny + 1), cudaMemcpyHostToDevice, c->stream));
  CK(c, cudaMemcpyAsync(coords + nx + ny + 2, zs, sizeof(double) * (nz + 1), cudaMemcpyHostToDevice, c->stream));
  CK(c, launch_box(nx, ny, nz, W, coords, coords + nx + 1, coords + nx + ny + 2, c->cs, c->stream));
  std::vector<int32_t> btype(NB, LFM_ZERO_GRADIENT);
  int rc;
  if ((rc = h2d(c, Y.btype, btype.data(), NB))) return rc;
  CK(c, cudaMemsetAsync(c->ws + Y.bDT, 0, sizeof(double) * NB, c->stream));
  CK(c, cudaMemsetAsync(c->ws + Y.bval, 0, sizeof(double) * NB, c->stream));
  const size_t WN = (size_t)W * N;
  if (WN > 0) {
    CK(c, cudaMemsetAsync(c->ws + Y.slot_coef, 0, sizeof(double) * WN, c->stream));
    if (has32) CK(c, cudaMemsetAsync(c->ws + Y.slot_coef32, 0, sizeof(float) * WN, c->stream));
  }
  CK(c, cudaMemsetAsync(c->ws + Y.DT, 0, sizeof(double) * (F > 0 ? F : 1), c->stream));
  c->cs.DT_is_uniform = 1;
  c->cs.DT_uniform = 0.0;
  CK(c, cudaMemsetAsync(c->ws + Y.x, 0, sizeof(double) * N, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  c->dt = 1.0;
  c->opts = lfm_solver_opts{1e-6, 0.0, 1000, 0, has64 ? LFM_FP64 : LFM_MIXED};
  if ((rc = refresh_vdt(c))) return rc;
  c->uploaded = true;
  c->ctas = c->threads = 0;
  return choose_launch(c);
}

size_t lfm_workspace_bytes_box(int32_t nx, int32_t ny, int32_t nz, int32_t precision) {
  int32_t N, F, NB, W;
  if (lfm_box_counts(nx, ny, nz, &N, &F, &NB, &W) != LFM_OK) return 0;
  precision = layout_kind(precision);
  return make_layout(N, F, NB, W, precision).total;
}

size_t lfm_workspace_bytes_shared(const lfm_ctx* src, int32_t precision) {
  if (!src || !src->uploaded) return 0;
  precision = layout_kind(precision);
  const lfm_ctx* root = src->mesh_src ? src->mesh_src : src;
  return make_layout(src->N, src->F, src->NB, src->W, precision, true, root->has_geom).total;
}

int lfm_upload_mesh_shared(lfm_ctx* c, lfm_ctx* src) {
  if (!c || !src) return fail_free(LFM_EINVAL, "context is NULL");
  if (c == src) return fail(c, LFM_EINVAL, "a context cannot share its own mesh");
  if (c->uploaded || c->n_sharers > 0) return fail(c, LFM_ESTATE, "the context already has a mesh");
  if (!src->uploaded) return fail(c, LFM_ESTATE, "the source context has no mesh");
  if (src->device != c->device) return fail(c, LFM_EINVAL, "the source context lives on another device");
  lfm_ctx* root = src->mesh_src ? src->mesh_src : src;
  DeviceGuard g(c->device);
  const int kind = c->ws_bound ? c->ws_kind : kLayoutBoth;
  const Layout use = make_layout(root->N, root->F, root->NB, root->W, kind, true, root->has_geom);
  const bool has64 = kind_has64(kind), has32 = kind_has32(kind), hasdf = kind_hasdf(kind);
  if (c->ws_bound) {
    if (c->ws_bytes < use.total) return fail(c, LFM_ENOMEM, "workspace has %zu bytes, needs %zu", c->ws_bytes, use.total);
  } else {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, use.total);
    if (e != cudaSuccess) return fail(c, LFM_ENOMEM, "device allocation of %zu bytes failed: %s", use.total, cudaGetErrorString(e));
    c->ws = static_cast<char*>(p);
    c->ws_bytes = use.total;
    c->ws_owned = true;
  }
  c->mesh_src = root;
  root->n_sharers++;
  c->lay = use;
  c->mean_V = root->mean_V;
  c->N = root->N;
  c->F = root->F;
  c->NB = root->NB;
  c->W = root->W;
  c->has64 = has64;
  c->has32 = has32;
  c->hasdf = hasdf;
  c->df_dirty = true;
  c->coef_dirty = true;
  c->has_geom = root->has_geom;
  c->ops_dirty = root->has_geom;
  c->n_corr = 0;
  c->has_Su = c->has_Sp = false;
  c->n_patches = root->n_patches;
  c->patch_start = root->patch_start;
  c->patch_size = root->patch_size;
  c->patch_type.assign(root->n_patches, LFM_ZERO_GRADIENT);
  bind_pointers(c);
  if (int e = invalidate_split(c)) return e;
  const int32_t N = c->N, F = c->F, NB = c->NB;
  const Layout& Y = c->lay;
  const size_t WN = (size_t)c->W * N;
  std::vector<int32_t> btype(NB > 0 ? NB : 1, LFM_ZERO_GRADIENT);
  int rc;
  if ((rc = h2d(c, Y.btype, btype.data(), NB))) return rc;
  CK(c, cudaMemsetAsync(c->ws + Y.bDT, 0, sizeof(double) * (NB > 0 ? NB : 1), c->stream));
  CK(c, cudaMemsetAsync(c->ws + Y.bval, 0, sizeof(double) * (NB > 0 ? NB : 1), c->stream));
  if (WN > 0) {
    CK(c, cudaMemsetAsync(c->ws + Y.slot_coef, 0, sizeof(double) * WN, c->stream));
    if (has32) CK(c, cudaMemsetAsync(c->ws + Y.slot_coef32, 0, sizeof(float) * WN, c->stream));
  }
  CK(c, cudaMemsetAsync(c->ws + Y.DT, 0, sizeof(double) * (F > 0 ? F : 1), c->stream));
  c->cs.DT_is_uniform = 1;
  c->cs.DT_uniform = 0.0;
  CK(c, cudaMemsetAsync(c->ws + Y.x, 0, sizeof(double) * N, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  c->dt = 1.0;
  c->opts = lfm_solver_opts{1e-6, 0.0, 1000, 0, has64 ? LFM_FP64 : LFM_MIXED};
  if ((rc = refresh_vdt(c))) return rc;
  c->uploaded = true;
  c->ctas = c->threads = 0;
  return choose_launch(c);
}

int lfm_fill_field(lfm_ctx* c, double value) {
  int rc = need_uploaded(c);
  if (rc) return rc;
  if (!std::isfinite(value)) return fail(c, LFM_EINVAL, "value must be finite");
  DeviceGuard g(c->device);
  if ((rc = invalidate_split(c))) return rc;
  CK(c, launch_fill(c->cs.x, c->N, value, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  return LFM_OK;
}

int lfm_set_diffusivity(lfm_ctx* c, double uniform, const double* DT_faces, const double* DT_bfaces) {
  int rc = need_uploaded(c);
  if (rc) return rc;
  if ((rc = invalidate_seed(c))) return rc;
  if (!(std::isfinite(uniform) && uniform >= 0)) return fail(c, LFM_EINVAL, "uniform DT must be finite and >= 0");
  for (int32_t f = 0; DT_faces && f < c->F; ++f)
    if (!(std::isfinite(DT_faces[f]) && DT_faces[f] >= 0)) return fail(c, LFM_EINVAL, "DT_faces[%d] must be finite and >= 0", f);
  for (int32_t b = 0; DT_bfaces && b < c->NB; ++b)
    if (!(std::isfinite(DT_bfaces[b]) && DT_bfaces[b] >= 0)) return fail(c, LFM_EINVAL, "DT_bfaces[%d] must be finite and >= 0", b);
  DeviceGuard g(c->device);
  if (DT_faces) {
    if ((rc = h2d(c, c->lay.DT, DT_faces, c->F))) return rc;
    c->cs.DT_is_uniform = 0;
  } else {
    CK(c, launch_fill(const_cast<double*>(c->cs.DT), c->F, uniform, c->stream));
    c->cs.DT_is_uniform = 1;
    c->cs.DT_uniform = uniform;
  }
  if (DT_bfaces) {
    if ((rc = h2d(c, c->lay.bDT, DT_bfaces, c->NB))) return rc;
  } else {
    CK(c, launch_fill(const_cast<double*>(c->cs.bDT), c->NB, uniform, c->stream));
  }
  CK(c, cudaStreamSynchronize(c->stream));
  c->ops_dirty = true;
  c->df_dirty = true;
  c->coef_dirty = true;
  return LFM_OK;
}

int lfm_set_diffusivity_cells(lfm_ctx* c, const double* DT_cells, const double* weights) {
  int rc = need_uploaded(c);
  if (rc) return rc;
  if ((rc = invalidate_seed(c))) return rc;
  if (!DT_cells) return fail(c, LFM_EINVAL, "DT_cells is NULL");
  if (!weights && !c->has_geom) return fail(c, LFM_EINVAL, "weights needed (the mesh has no geometry)");
  for (int32_t i = 0; i < c->N; ++i)
    if (!(std::isfinite(DT_cells[i]) && DT_cells[i] >= 0)) return fail(c, LFM_EINVAL, "DT_cells[%d] must be finite and >= 0", i);
  for (int32_t f = 0; weights && f < c->F; ++f)
    if (!(std::isfinite(weights[f]) && weights[f] >= 0 && weights[f] <= 1))
      return fail(c, LFM_EINVAL, "weights[%d] not in [0, 1]", f);
  DeviceGuard g(c->device);
  double* tmp = nullptr;
  const size_t n = (size_t)c->N + (weights ? (size_t)c->F : 0);
  cudaError_t e = cudaMalloc(&tmp, sizeof(double) * (n > 0 ? n : 1));
  if (e != cudaSuccess) return fail(c, LFM_ENOMEM, "staging buffer: %s", cudaGetErrorString(e));
  e = cudaMemcpyAsync(tmp, DT_cells, sizeof(double) * c->N, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess && weights)
    e = cudaMemcpyAsync(tmp + c->N, weights, sizeof(double) * c->F, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = launch_dt_cells(c->cs, tmp, weights ? tmp + c->N : c->cs.fw, const_cast<double*>(c->cs.DT),
                        const_cast<double*>(c->cs.bDT), c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  cudaFree(tmp);
  if (e != cudaSuccess) return cuda_fail(c, e, "lfm_set_diffusivity_cells");
  c->cs.DT_is_uniform = 0;
  c->ops_dirty = true;
  c->df_dirty = true;
  c->coef_dirty = true;
  return LFM_OK;
}

int lfm_set_source(lfm_ctx* c, const double* Su, const double* Sp) {
  int rc = need_uploaded(c);
  if (rc) return rc;
  if ((rc = invalidate_seed(c))) return rc;
  if (c->pending_steps > 0) return fail(c, LFM_ESTATE, "an advance is pending");
  for (int32_t i = 0; Su && i < c->N; ++i)
    if (!std::isfinite(Su[i])) return fail(c, LFM_EINVAL, "Su[%d] not finite", i);
  for (int32_t i = 0; Sp && i < c->N; ++i)
    if (!std::isfinite(Sp[i])) return fail(c, LFM_EINVAL, "Sp[%d] not finite", i);
  DeviceGuard g(c->device);
  double* tmp = nullptr;
  if (Su || Sp) {
    cudaError_t e = cudaMalloc(&tmp, sizeof(double) * c->N);
    if (e != cudaSuccess) return fail(c, LFM_ENOMEM, "staging buffer: %s", cudaGetErrorString(e));
  }
  const double* src[2] = {Su, Sp};
  const size_t off[2] = {c->lay.vSu, c->lay.vSp};
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
    if (!src[k]) continue;
    e = cudaMemcpyAsync(tmp, src[k], sizeof(double) * c->N, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = launch_times_volume(c->cs, tmp, reinterpret_cast<double*>(c->ws + off[k]), c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  }
  if (tmp) cudaFree(tmp);
  if (e != cudaSuccess) return cuda_fail(c, e, "lfm_set_source");
  c->has_Su = Su != nullptr;
  c->has_Sp = Sp != nullptr;
  bind_pointers(c);
  return LFM_OK;
}

int lfm_set_patch(lfm_ctx* c, int32_t patch, int32_t type, const double* values, double uniform) {
  int rc = need_uploaded(c);
  if (rc) return rc;
  if ((rc = invalidate_seed(c))) return rc;
  if (patch < 0 || patch >= c->n_patches) return fail(c, LFM_EINVAL, "patch %d out of range", patch);
  if (type != LFM_FIXED_VALUE && type != LFM_ZERO_GRADIENT) return fail(c, LFM_EINVAL, "unknown patch type %d", type);
  const int32_t n = c->patch_size[patch], s = c->patch_start[patch];
  std::vector<double> vals(n > 0 ? n : 1, uniform);
  if (type == LFM_FIXED_VALUE) {
    if (values) std::copy(values, values + n, vals.begin());
    for (int32_t i = 0; i < n; ++i)
      if (!std::isfinite(vals[i])) return fail(c, LFM_EINVAL, "patch %d value %d not finite", patch, i);
  }
  std::vector<int32_t> types(n > 0 ? n : 1, type);
  DeviceGuard g(c->device);
  if ((rc = h2d(c, c->lay.btype + 4 * (size_t)s, types.data(), n))) return rc;
  if (type == LFM_FIXED_VALUE && (rc = h2d(c, c->lay.bval + 8 * (size_t)s, vals.data(), n))) return rc;
  CK(c, cudaStreamSynchronize(c->stream));
  c->patch_type[patch] = type;
  c->ops_dirty = true;
  return LFM_OK;
}

int lfm_set_time_step(lfm_ctx* c, double dt) {
  int rc = need_uploaded(c);
  if (rc) return rc;
  if ((rc = invalidate_seed(c))) return rc;
  if (!(std::isfinite(dt) && dt > 0)) return fail(c, LFM_EINVAL, "dt must be finite and > 0");
  if (c->pending_steps > 0 || ctx_batch_pending(c)) return fail(c, LFM_ESTATE, "an advance is pending");
  c->dt = dt;
  DeviceGuard g(c->device);
  return refresh_vdt(c);
}

int lfm_set_solver(lfm_ctx* c, const lfm_solver_opts* o) {
  int rc = need_uploaded(c);
  if (rc) return rc;
  if ((rc = invalidate_seed(c))) return rc;
  if (!o) return fail(c, LFM_EINVAL, "opts is NULL");
  if (!(std::isfinite(o->tol) && o->tol >= 0) || !(std::isfinite(o->rel_tol) && o->rel_tol >= 0) ||
      o->max_iter < 1 || o->min_iter < 0 || o->min_iter > o->max_iter ||
      (o->precision != LFM_FP64 && o->precision != LFM_MIXED && o->precision != LFM_DF64))
    return fail(c, LFM_EINVAL, "invalid solver options");
  if ((o->precision == LFM_FP64 && !c->has64) || (o->precision == LFM_MIXED && !c->has32) ||
      (o->precision == LFM_DF64 && !(c->hasdf && c->has64)))
    return fail(c, LFM_ENOMEM, "the workspace was laid out without the %s solver buffers",
                o->precision == LFM_FP64 ? "FP64" : (o->precision == LFM_MIXED ? "mixed-precision" : "df64"));
  if (o->precision == LFM_DF64 && c->has_geom && !c->cs.gE2)
    return fail(c, LFM_ENOMEM, "the workspace was laid out without the df64 general-geometry buffers");
  const bool launch_changes = o->precision != c->opts.precision;
  c->opts = *o;
  if (launch_changes) return choose_launch(c);
  return LFM_OK;
}

int lfm_set_nonorth_correctors(lfm_ctx* c, int32_t n_corr) {
  int rc = need_uploaded(c);
  if (rc) return rc;
  if ((rc = invalidate_seed(c))) return rc;
  if (n_corr < 0 || n_corr > 64) return fail(c, LFM_EINVAL, "n_corr must be in [0, 64] (got %d)", n_corr);
  if (c->pending_steps > 0) return fail(c, LFM_ESTATE, "an advance is pending");
  c->n_corr = n_corr;
  return LFM_OK;
}

int lfm_grad(lfm_ctx* c, double* grad, double* bgrad) {
  int rc = need_uploaded(c);
  if (rc) return rc;
  if (!c->has_geom) return fail(c, LFM_ESTATE, "the mesh was uploaded without general geometry");
  if (!grad) return fail(c, LFM_EINVAL, "grad is NULL");
  if (c->pending_steps > 0) return fail(c, LFM_ESTATE, "an advance is pending");
  DeviceGuard g(c->device);
  refresh_case(c);
  if ((rc = refresh_ops(c))) return rc;
  double* bdev = nullptr;
  if (bgrad && c->NB > 0) {
    cudaError_t e = cudaMalloc(&bdev, sizeof(double) * 3 * (size_t)c->NB);
    if (e != cudaSuccess) return fail(c, LFM_ENOMEM, "boundary gradient buffer: %s", cudaGetErrorString(e));
  }
  const size_t N = (size_t)c->N;
  std::vector<double> soa(3 * N);
  cudaError_t e = launch_grad(c->cs, bdev, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(soa.data(), c->cs.grad, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess && bdev)
    e = cudaMemcpyAsync(bgrad, bdev, sizeof(double) * 3 * (size_t)c->NB, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (bdev) cudaFree(bdev);
  if (e != cudaSuccess) return cuda_fail(c, e, "lfm_grad");
  for (size_t i = 0; i < N; ++i)
    for (int d = 0; d < 3; ++d) grad[3 * i + d] = soa[d * N + i];  // cell-major for the caller
  return LFM_OK;
}

int lfm_set_field(lfm_ctx* c, const double* T) {
  int rc = need_uploaded(c);
  if (rc) return rc;
  if (!T) return fail(c, LFM_EINVAL, "T is NULL");
  DeviceGuard g(c->device);
  if ((rc = invalidate_split(c))) return rc;
  CK(c, cudaMemcpyAsync(c->cs.x, T, sizeof(double) * c->N, cudaMemcpyHostToDevice, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  return LFM_OK;
}

int lfm_set_field_device(lfm_ctx* c, const double* T_dev) {
  int rc = need_uploaded(c);
  if (rc) return rc;
  if (!T_dev) return fail(c, LFM_EINVAL, "T_dev is NULL");
  DeviceGuard g(c->device);
  if ((rc = invalidate_split(c))) return rc;
  CK(c, cudaMemcpyAsync(c->cs.x, T_dev, sizeof(double) * c->N, cudaMemcpyDeviceToDevice, c->stream));
  return LFM_OK;
}

int lfm_advance_async(lfm_ctx* c, int32_t n_steps) {
  int rc = need_uploaded(c);
  if (rc) return rc;
  if (n_steps < 0) return fail(c, LFM_EINVAL, "n_steps must be >= 0");
  if (c->pending_steps > 0) return fail(c, LFM_ESTATE, "an advance is already pending");
  if (n_steps == 0) return LFM_OK;
  DeviceGuard g(c->device);
  c->stats_acc.clear();
  for (int k = 0; k < kPhases; ++k) c->phase_ms[k] = 0.0;
  c->staged_passes = 0;
  const int first = n_steps < kStatsCap ? n_steps : kStatsCap;
  if ((rc = enqueue_chunk(c, first, kModeSteps))) return rc;
  c->pending_steps = first;
  c->pending_remaining = n_steps - first;
  return LFM_OK;
}

int lfm_query(lfm_ctx* c) {
  if (!c) return fail_free(LFM_EINVAL, "context is NULL");
  if (c->pending_steps == 0) return LFM_OK;
  if (c->pending_remaining > 0) return 1;
  DeviceGuard g(c->device);
  cudaError_t e = cudaEventQuery(c->done);
  if (e == cudaErrorNotReady) return 1;
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaEventQuery");
  return LFM_OK;
}

int lfm_finish(lfm_ctx* c, lfm_step_stats* out, int32_t n) {
  if (!c) return fail_free(LFM_EINVAL, "context is NULL");
  DeviceGuard g(c->device);
  int rc = LFM_OK;
  while (c->pending_steps > 0) {
    rc = collect_chunk(c, c->pending_steps);
    c->pending_steps = 0;
    if (rc != LFM_OK) {
      c->pending_remaining = 0;
      break;
    }
    if (c->pending_remaining > 0) {
      const int next = c->pending_remaining < kStatsCap ? c->pending_remaining : kStatsCap;
      if ((rc = enqueue_chunk(c, next, kModeSteps))) {
        c->pending_remaining = 0;
        break;
      }
      c->pending_steps = next;
      c->pending_remaining -= next;
    }
  }
  if (out) {
    const int32_t m = (int32_t)c->stats_acc.size() < n ? (int32_t)c->stats_acc.size() : n;
    for (int32_t i = 0; i < m; ++i) out[i] = c->stats_acc[i];
  }
  return rc;
}

int lfm_advance(lfm_ctx* c, int32_t n_steps, lfm_step_stats* out) {
  int rc = lfm_advance_async(c, n_steps);
  if (rc != LFM_OK) return rc;
  return lfm_finish(c, out, n_steps);
}

int lfm_get_field(lfm_ctx* c, double* T_out, double* T_boundary) {
  int rc = need_uploaded(c);
  if (rc) return rc;
  if (!T_out) return fail(c, LFM_EINVAL, "T_out is NULL");
  DeviceGuard g(c->device);
  CK(c, cudaMemcpyAsync(T_out, c->cs.x, sizeof(double) * c->N, cudaMemcpyDeviceToHost, c->stream));
  if (T_boundary && c->NB > 0) {
    double* Tb = reinterpret_cast<double*>(c->ws + c->lay.Tb);
    CK(c, launch_boundary_values(c->cs, Tb, c->stream));
    CK(c, cudaMemcpyAsync(T_boundary, Tb, sizeof(double) * c->NB, cudaMemcpyDeviceToHost, c->stream));
  }
  CK(c, cudaStreamSynchronize(c->stream));
  return LFM_OK;
}

int lfm_field_device_ptr(lfm_ctx* c, double** T_dev) {
  int rc = need_uploaded(c);
  if (rc) return rc;
  if (!T_dev) return fail(c, LFM_EINVAL, "T_dev is NULL");
  *T_dev = c->cs.x;
  return LFM_OK;
}

int lfm_get_matrix(lfm_ctx* c, double* diag, double* upper, double* source) {
  int rc = need_uploaded(c);
  if (rc) return rc;
  if ((rc = invalidate_seed(c))) return rc;
  if (!diag || !source || (c->F > 0 && !upper)) return fail(c, LFM_EINVAL, "output arrays missing");
  if (c->pending_steps > 0) return fail(c, LFM_ESTATE, "an advance is pending");
  DeviceGuard g(c->device);
  if ((rc = enqueue_chunk(c, 1, kModeAssembleOnly))) return rc;
  c->stats_acc.clear();
  CK(c, cudaEventSynchronize(c->done));
  if (*c->h_status != 0) return fail(c, LFM_ETIMEOUT, "assembly launch failed with device status %d", *c->h_status);
  CK(c, cudaMemcpyAsync(diag, c->cs.diag, sizeof(double) * c->N, cudaMemcpyDeviceToHost, c->stream));
  if (c->F > 0) CK(c, cudaMemcpyAsync(upper, c->cs.upper, sizeof(double) * c->F, cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaMemcpyAsync(source, c->cs.src, sizeof(double) * c->N, cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  return LFM_OK;
}

int lfm_get_addressing(lfm_ctx* c, int32_t* slot_other, int32_t* slot_face, uint32_t* face_slots, int32_t* b_start,
                       int32_t* b_face) {
  int rc = need_uploaded(c);
  if (rc) return rc;
  DeviceGuard g(c->device);
  const size_t WN = (size_t)c->W * c->N;
  if (slot_other && WN) CK(c, cudaMemcpyAsync(slot_other, c->cs.slot_other, 4 * WN, cudaMemcpyDeviceToHost, c->stream));
  if (slot_face && WN) CK(c, cudaMemcpyAsync(slot_face, c->cs.slot_face, 4 * WN, cudaMemcpyDeviceToHost, c->stream));
  if (face_slots && c->F)
    CK(c, cudaMemcpyAsync(face_slots, c->cs.face_slots, 8 * (size_t)c->F, cudaMemcpyDeviceToHost, c->stream));
  if (b_start) CK(c, cudaMemcpyAsync(b_start, c->cs.b_start, 4 * ((size_t)c->N + 1), cudaMemcpyDeviceToHost, c->stream));
  if (b_face && c->NB) CK(c, cudaMemcpyAsync(b_face, c->cs.b_face, 4 * (size_t)c->NB, cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  return LFM_OK;
}

int lfm_get_phase_times(lfm_ctx* c, double* ms) {
  int rc = need_uploaded(c);
  if (rc) return rc;
  if (!ms) return fail(c, LFM_EINVAL, "ms is NULL");
  for (int k = 0; k < kPhases; ++k) ms[k] = c->phase_ms[k];
  return LFM_OK;
}

int lfm_get_launch(lfm_ctx* c, int32_t* ctas, int32_t* threads) {
  int rc = need_uploaded(c);
  if (rc) return rc;
  int e = 0;
  Launch L = current_launch(c, e);
  if (ctas) *ctas = L.ctas;
  if (threads) *threads = L.threads;
  return e ? fail(c, LFM_ECUDA, "no co-resident CTA fits") : LFM_OK;
}

int lfm_set_launch(lfm_ctx* c, int32_t ctas, int32_t threads) {
  int rc = need_uploaded(c);
  if (rc) return rc;
  if ((rc = invalidate_seed(c))) return rc;
  if (threads > 0 && threads != 256 && threads != 512 && threads != 1024)
    return fail(c, LFM_EINVAL, "threads must be 256, 512 or 1024");
  c->ctas = ctas > 0 ? ctas : 0;
  c->threads = threads > 0 ? threads : 0;
  return LFM_OK;
}

int lfm_set_barrier_timeout(lfm_ctx* c, uint64_t ns) {
  if (!c) return fail_free(LFM_EINVAL, "context is NULL");
  if (ns == 0) return fail(c, LFM_EINVAL, "timeout must be > 0");
  c->timeout_ns = ns;
  return LFM_OK;
}

int lfm_checked_build(void) { return kCheckedBuild ? 1 : 0; }

int lfm_debug_check_inject(lfm_ctx* c, int32_t site) {
  if (!c) return fail_free(LFM_EINVAL, "context is NULL");
  if (!kCheckedBuild) return fail(c, LFM_ESTATE, "index checks are compiled only into the checked build");
  if (site < 1 || site > 4) return fail(c, LFM_EINVAL, "check site %d is not one of 1..4", site);
  DeviceGuard g(c->device);
  check_inject_step(site, c->stream);
  check_inject_batch(site, c->stream);
  return LFM_OK;
}

int lfm_debug_skip_arrival(lfm_ctx* c, int32_t cta) {
  if (!c) return fail_free(LFM_EINVAL, "context is NULL");
  c->skip_cta = cta >= 0 ? cta : -1;
  return LFM_OK;
}

int lfm_debug_skip_stage_copy(lfm_ctx* c, int32_t cta) {
  if (!c) return fail_free(LFM_EINVAL, "context is NULL");
  c->skip_copy_cta = cta >= 0 ? cta : -1;
  return LFM_OK;
}

int lfm_debug_staged_passes(lfm_ctx* c, int64_t* n) {
  if (!c) return fail_free(LFM_EINVAL, "context is NULL");
  if (!n) return fail(c, LFM_EINVAL, "n is NULL");
  *n = c->staged_passes;
  return LFM_OK;
}

int lfm_debug_stage_rows(lfm_ctx* c, int32_t on) {
  if (!c) return fail_free(LFM_EINVAL, "context is NULL");
  c->stage_rows = on != 0 ? 1 : 0;
  return LFM_OK;
}

int lfm_destroy(lfm_ctx* c) {
  if (!c) return LFM_OK;
  if (c->batch) return fail(c, LFM_ESTATE, "remove the context from its batch first");
  if (c->n_sharers > 0) return fail(c, LFM_ESTATE, "%d contexts still use this context's mesh", c->n_sharers);
  if (c->mesh_src) c->mesh_src->n_sharers--;
  {
    DeviceGuard g(c->device);
    if (c->pending_steps > 0 && c->done) cudaEventSynchronize(c->done);
    if (c->ws_owned && c->ws) cudaFree(c->ws);
    if (c->h_stats) cudaFreeHost(c->h_stats);
    if (c->h_status) cudaFreeHost(c->h_status);
    if (c->h_phase) cudaFreeHost(c->h_phase);
    if (c->done) cudaEventDestroy(c->done);
  }
  delete c;
  return LFM_OK;
}

const char* lfm_last_error(const lfm_ctx* c) {
  if (c) return c->err.c_str();
  return g_last_error.c_str();
}


}  // extern "C"

// ======================================================================================
// Batched form
// ======================================================================================

struct lfm_batch {
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t capture_stream = nullptr;
  std::string err;
  std::vector<lfm_ctx*> slots;      // case id -> member (nullptr once removed)
  std::vector<double> est_iters;    // per case id: PCG iterations of its last step
  std::vector<int32_t> status;      // per case id: status of the last advance
  std::vector<int32_t> last_iters;  // per case id: PCG iterations of its last step (-1: none)
  std::vector<int32_t> steps_run;   // per case id: steps run by the last advance
  std::vector<int32_t> iters_run;   // per case id: PCG iterations summed over those steps
  std::vector<int32_t> order;       // compact index of the last advance -> case id
  int threads = 512;
  int cpt[3] = {4, 8, 16};          // cells per thread by size class
  uint64_t timeout_ns = 10000000000ull;
  // device buffers, library-owned
  int cap = 0;
  CaseDev* d_cases = nullptr;
  int32_t* d_job_case = nullptr;
  int32_t* d_job_start = nullptr;
  BatchHeader* d_hdr = nullptr;
  int32_t* d_case_step = nullptr;
  int32_t* d_status = nullptr;
  int32_t* d_iters = nullptr;
  int32_t* d_cap = nullptr;
  int32_t* d_steps = nullptr;
  int32_t* d_iters_sum = nullptr;
  // pinned staging
  CaseDev* h_cases = nullptr;
  int32_t* h_job_case = nullptr;
  int32_t* h_job_start = nullptr;
  BatchHeader* h_hdr = nullptr;
  int32_t* h_status = nullptr;
  int32_t* h_iters = nullptr;
  int32_t* h_cap = nullptr;
  int32_t* h_steps = nullptr;
  int32_t* h_iters_sum = nullptr;
  cudaEvent_t done = nullptr;
  int pending = 0;
  int n_active = 0;
  // captured one-step graph
  cudaGraphExec_t gexec = nullptr;
  int g_threads = 0, g_W = -1, g_ctas = 0, g_form = -1, g_stage = -1;
  int stage_rows = 1;  // bulk-staged matrix rows where a pass supports them
  int last_ctas = 0, last_W = 6, last_form = kBatchAny;
};

namespace {

thread_local std::string g_batch_error;

}  // namespace

namespace {
bool ctx_batch_pending(const lfm_ctx* c) { return c->batch && c->batch->pending; }


int bfail(lfm_batch* b, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (b) b->err = buf;
  g_batch_error = buf;
  return code;
}

#define BCK(b, call)                                                                     \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) return bfail(b, LFM_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

int size_class(int32_t N) { return N < 32768 ? 0 : (N < 262144 ? 1 : 2); }

void free_buffers(lfm_batch* b) {
  cudaFree(b->d_cases);
  cudaFree(b->d_job_case);
  cudaFree(b->d_job_start);
  cudaFree(b->d_hdr);
  cudaFree(b->d_case_step);
  cudaFree(b->d_status);
  cudaFree(b->d_iters);
  cudaFree(b->d_cap);
  cudaFree(b->d_steps);
  cudaFree(b->d_iters_sum);
  cudaFreeHost(b->h_cases);
  cudaFreeHost(b->h_job_case);
  cudaFreeHost(b->h_job_start);
  cudaFreeHost(b->h_hdr);
  cudaFreeHost(b->h_status);
  cudaFreeHost(b->h_iters);
  cudaFreeHost(b->h_cap);
  cudaFreeHost(b->h_steps);
  cudaFreeHost(b->h_iters_sum);
  b->d_cases = nullptr;
  b->d_job_case = b->d_job_start = b->d_case_step = b->d_status = b->d_iters = nullptr;
  b->d_cap = b->d_steps = b->d_iters_sum = nullptr;
  b->h_cap = b->h_steps = b->h_iters_sum = nullptr;
  b->d_hdr = nullptr;
  b->h_cases = nullptr;
  b->h_job_case = b->h_job_start = b->h_status = b->h_iters = nullptr;
  b->h_hdr = nullptr;
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  b->gexec = nullptr;
  b->cap = 0;
}

int ensure_capacity(lfm_batch* b, int n) {
  if (n <= b->cap) return LFM_OK;
  int cap = b->cap ? b->cap : 64;
  while (cap < n) cap *= 2;
  free_buffers(b);
  BCK(b, cudaMalloc(&b->d_cases, sizeof(CaseDev) * cap));
  BCK(b, cudaMalloc(&b->d_job_case, sizeof(int32_t) * cap));
  BCK(b, cudaMalloc(&b->d_job_start, sizeof(int32_t) * (cap + 1)));
  BCK(b, cudaMalloc(&b->d_hdr, sizeof(BatchHeader)));
  BCK(b, cudaMalloc(&b->d_case_step, sizeof(int32_t) * cap));
  BCK(b, cudaMalloc(&b->d_status, sizeof(int32_t) * cap));
  BCK(b, cudaMalloc(&b->d_iters, sizeof(int32_t) * cap));
  BCK(b, cudaMalloc(&b->d_cap, sizeof(int32_t) * cap));
  BCK(b, cudaMalloc(&b->d_steps, sizeof(int32_t) * cap));
  BCK(b, cudaMalloc(&b->d_iters_sum, sizeof(int32_t) * cap));
  BCK(b, cudaMallocHost(&b->h_cases, sizeof(CaseDev) * cap));
  BCK(b, cudaMallocHost(&b->h_job_case, sizeof(int32_t) * cap));
  BCK(b, cudaMallocHost(&b->h_job_start, sizeof(int32_t) * (cap + 1)));
  BCK(b, cudaMallocHost(&b->h_hdr, sizeof(BatchHeader)));
  BCK(b, cudaMallocHost(&b->h_status, sizeof(int32_t) * cap));
  BCK(b, cudaMallocHost(&b->h_iters, sizeof(int32_t) * cap));
  BCK(b, cudaMallocHost(&b->h_cap, sizeof(int32_t) * cap));
  BCK(b, cudaMallocHost(&b->h_steps, sizeof(int32_t) * cap));
  BCK(b, cudaMallocHost(&b->h_iters_sum, sizeof(int32_t) * cap));
  b->cap = cap;
  return LFM_OK;
}

}  // namespace

extern "C" {

int lfm_batch_create(lfm_batch** out, int device, void* cuda_stream) {
  if (!out) return bfail(nullptr, LFM_EINVAL, "out is NULL");
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) return bfail(nullptr, LFM_ECUDA, "no CUDA device");
  if (device < 0 || device >= n) return bfail(nullptr, LFM_EINVAL, "device %d out of range", device);
  lfm_batch* b = new (std::nothrow) lfm_batch;
  if (!b) return bfail(nullptr, LFM_ENOMEM, "out of host memory");
  b->device = device;
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  DeviceGuard g(device);
  if (cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
    lfm_batch_destroy(b);
    return bfail(nullptr, LFM_ECUDA, "event or stream creation failed");
  }
  *out = b;
  return LFM_OK;
}

int lfm_batch_add(lfm_batch* b, lfm_ctx* c, int32_t* case_id) {
  if (!b || !c) return bfail(b, LFM_EINVAL, "batch or context is NULL");
  if (b->pending) return bfail(b, LFM_ESTATE, "an advance is pending");
  if (!c->uploaded) return bfail(b, LFM_ESTATE, "the context has no mesh");
  if (c->batch) return bfail(b, LFM_ESTATE, "the context already belongs to a batch");
  if (c->device != b->device) return bfail(b, LFM_EINVAL, "the context lives on device %d, the batch on %d", c->device, b->device);
  if (c->pending_steps) return bfail(b, LFM_ESTATE, "the context has a pending advance");
  int32_t id = -1;
  for (size_t i = 0; i < b->slots.size(); ++i)
    if (!b->slots[i]) {
      id = (int32_t)i;
      break;
    }
  if (id < 0) {
    id = (int32_t)b->slots.size();
    b->slots.push_back(nullptr);
    b->est_iters.push_back(5.0);
    b->status.push_back(0);
    b->last_iters.push_back(-1);
    b->steps_run.push_back(0);
    b->iters_run.push_back(0);
  }
  b->slots[id] = c;
  b->est_iters[id] = 5.0;
  b->status[id] = 0;
  b->last_iters[id] = -1;
  b->steps_run[id] = 0;
  b->iters_run[id] = 0;
  c->batch = b;
  if (case_id) *case_id = id;
  return LFM_OK;
}

int lfm_batch_remove(lfm_batch* b, int32_t id) {
  if (!b) return bfail(nullptr, LFM_EINVAL, "batch is NULL");
  if (b->pending) return bfail(b, LFM_ESTATE, "an advance is pending");
  if (id < 0 || id >= (int32_t)b->slots.size() || !b->slots[id]) return bfail(b, LFM_EINVAL, "no case %d", id);
  b->slots[id]->batch = nullptr;
  b->slots[id] = nullptr;
  return LFM_OK;
}

int lfm_batch_size(const lfm_batch* b) {
  if (!b) return 0;
  int n = 0;
  for (lfm_ctx* c : b->slots) n += c != nullptr;
  return n;
}

int lfm_batch_debug_stage_rows(lfm_batch* b, int32_t on) {
  if (!b) return fail_free(LFM_EINVAL, "batch is NULL");
  b->stage_rows = on != 0 ? 1 : 0;
  return LFM_OK;
}

int lfm_batch_set_launch(lfm_batch* b, int32_t threads, const int32_t* cells_per_thread) {
  if (!b) return bfail(nullptr, LFM_EINVAL, "batch is NULL");
  if (threads != 256 && threads != 512) return bfail(b, LFM_EINVAL, "threads must be 256 or 512");
  if (cells_per_thread)
    for (int k = 0; k < 3; ++k)
      if (cells_per_thread[k] < 1 || cells_per_thread[k] > (1 << 20)) return bfail(b, LFM_EINVAL, "cells per thread out of range");
  b->threads = threads;
  if (cells_per_thread)
    for (int k = 0; k < 3; ++k) b->cpt[k] = cells_per_thread[k];
  return LFM_OK;
}

int lfm_batch_get_launch(lfm_batch* b, int32_t* ctas, int32_t* threads, int32_t* cells_per_thread) {
  if (!b) return bfail(nullptr, LFM_EINVAL, "batch is NULL");
  DeviceGuard g(b->device);
  if (ctas) *ctas = max_coresident_batch_ctas(b->threads, b->last_W, b->last_form, b->device);
  if (threads) *threads = b->threads;
  if (cells_per_thread)
    for (int k = 0; k < 3; ++k) cells_per_thread[k] = b->cpt[k];
  return LFM_OK;
}

int lfm_batch_set_barrier_timeout(lfm_batch* b, uint64_t ns) {
  if (!b || ns == 0) return bfail(b, LFM_EINVAL, "bad timeout");
  b->timeout_ns = ns;
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  b->gexec = nullptr;
  return LFM_OK;
}

int lfm_batch_advance_async(lfm_batch* b, int32_t n_steps, int32_t use_graph) {
  return lfm_batch_advance_capped_async(b, n_steps, use_graph, nullptr, 0);
}

int lfm_batch_advance_capped_async(lfm_batch* b, int32_t n_steps, int32_t use_graph, const int32_t* caps,
                                   int32_t n_caps) {
  if (!b) return bfail(nullptr, LFM_EINVAL, "batch is NULL");
  if (b->pending) return bfail(b, LFM_ESTATE, "an advance is pending");
  if (n_steps < 0 || n_steps > kStatsCap) return bfail(b, LFM_EINVAL, "n_steps must be in [0, %d]", kStatsCap);
  if (n_caps < 0 || (n_caps > 0 && !caps)) return bfail(b, LFM_EINVAL, "caps is NULL or n_caps < 0");
  for (int32_t i = 0; i < n_caps; ++i)
    if (caps[i] < 0) return bfail(b, LFM_EINVAL, "caps[%d] = %d is negative", i, caps[i]);
  DeviceGuard g(b->device);
  b->order.clear();
  for (size_t i = 0; i < b->slots.size(); ++i)
    if (b->slots[i]) b->order.push_back((int32_t)i);
  const int n = (int)b->order.size();
  b->n_active = n;
  if (n == 0 || n_steps == 0) return LFM_OK;
  int rc = ensure_capacity(b, n);
  if (rc) return rc;
  int W = 6, form = kBatchAny;
  for (int i = 0; i < n; ++i) {
    lfm_ctx* c = b->slots[b->order[i]];
    if (c->pending_steps) return bfail(b, LFM_ESTATE, "case %d has a pending advance of its own", b->order[i]);
    refresh_case(c);
    if (refresh_ops(c) != LFM_OK) return bfail(b, LFM_ECUDA, "case %d: operator rebuild failed", b->order[i]);
    if ((c->opts.precision == LFM_FP64 && !c->has64) || (c->opts.precision == LFM_MIXED && !c->has32) ||
        (c->opts.precision == LFM_DF64 && !(c->hasdf && c->has64)))
      return bfail(b, LFM_ENOMEM, "case %d has no buffers for its precision", b->order[i]);
    if (refresh_coef(c) != LFM_OK || refresh_df(c) != LFM_OK)
      return bfail(b, LFM_ECUDA, "case %d: coefficient set-up failed", b->order[i]);
    b->h_cases[i] = c->cs;
    if (c->W != 6) W = 0;
    const int p = c->opts.precision;
    const int f = p == LFM_FP64 ? kBatchFp64 : p == LFM_DF64 ? kBatchDf64 : kBatchAny;
    form = i == 0 ? f : (form == f ? form : kBatchAny);
  }
  const int ctas = max_coresident_batch_ctas(b->threads, W, form, b->device);
  if (ctas <= 0) return bfail(b, LFM_ECUDA, "no co-resident CTA fits the batch kernel");
  // jobs: team sizes from the size classes, longest (estimated) job first
  std::vector<int> k(n), idx(n);
  std::vector<double> t(n);
  for (int i = 0; i < n; ++i) {
    const int32_t N = b->h_cases[i].N;
    const int64_t per_cta = (int64_t)b->threads * b->cpt[size_class(N)];
    int64_t kk = (N + per_cta - 1) / per_cta;
    if (kk < 1) kk = 1;
    if (kk > ctas) kk = ctas;
    k[i] = (int)kk;
    const int32_t id = b->order[i];
    const int32_t run = (id < n_caps && caps[id] < n_steps) ? caps[id] : n_steps;
    b->h_cap[i] = run;
    t[i] = (double)N * (b->est_iters[id] + 2.0) * (double)run / (double)kk;
    idx[i] = i;
  }
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int c) { return t[a] > t[c]; });
  int32_t tickets = 0;
  for (int j = 0; j < n; ++j) {
    b->h_job_case[j] = idx[j];
    b->h_job_start[j] = tickets;
    tickets += k[idx[j]];
  }
  b->h_job_start[n] = tickets;
  b->h_hdr->n_jobs = n;
  b->h_hdr->n_tickets = tickets;
  b->h_hdr->ticket = 0;
  b->h_hdr->pad = 0;
  BCK(b, cudaMemcpyAsync(b->d_cases, b->h_cases, sizeof(CaseDev) * n, cudaMemcpyHostToDevice, b->stream));
  BCK(b, cudaMemcpyAsync(b->d_job_case, b->h_job_case, sizeof(int32_t) * n, cudaMemcpyHostToDevice, b->stream));
  BCK(b, cudaMemcpyAsync(b->d_job_start, b->h_job_start, sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice, b->stream));
  BCK(b, cudaMemcpyAsync(b->d_hdr, b->h_hdr, sizeof(BatchHeader), cudaMemcpyHostToDevice, b->stream));
  BCK(b, cudaMemcpyAsync(b->d_cap, b->h_cap, sizeof(int32_t) * n, cudaMemcpyHostToDevice, b->stream));
  BCK(b, launch_batch_prepare(b->d_cases, n, b->d_case_step, b->stream));

  BatchLaunch bl{};
  bl.cases = b->d_cases;
  bl.job_case = b->d_job_case;
  bl.job_start = b->d_job_start;
  bl.hdr = b->d_hdr;
  bl.case_step = b->d_case_step;
  bl.case_cap = b->d_cap;
  bl.launch.ctas = ctas;
  bl.launch.threads = b->threads;
  bl.launch.timeout_ns = b->timeout_ns;
  bl.launch.skip_cta = -1;
  bl.launch.stage_rows = b->stage_rows;
  bl.launch.skip_copy_cta = -1;
  bl.W = W;
  bl.form = form;
  b->last_ctas = ctas;
  b->last_W = W;
  b->last_form = form;
  if (use_graph) {
    if (!b->gexec || b->g_threads != b->threads || b->g_W != W || b->g_ctas != ctas || b->g_form != form ||
        b->g_stage != b->stage_rows) {
      if (b->gexec) cudaGraphExecDestroy(b->gexec);
      b->gexec = nullptr;
      cudaGraph_t graph = nullptr;
      BCK(b, cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal));
      cudaError_t le = launch_batch_steps(bl, 1, b->capture_stream);
      cudaError_t ce = cudaStreamEndCapture(b->capture_stream, &graph);
      if (le != cudaSuccess || ce != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return bfail(b, LFM_ECUDA, "capturing the batch step failed: %s / %s", cudaGetErrorString(le),
                     cudaGetErrorString(ce));
      }
      cudaError_t ie = cudaGraphInstantiate(&b->gexec, graph, 0);
      cudaGraphDestroy(graph);
      if (ie != cudaSuccess) return bfail(b, LFM_ECUDA, "instantiating the batch step graph failed: %s", cudaGetErrorString(ie));
      b->g_threads = b->threads;
      b->g_W = W;
      b->g_ctas = ctas;
      b->g_form = form;
      b->g_stage = b->stage_rows;
    }
    for (int s = 0; s < n_steps; ++s) BCK(b, cudaGraphLaunch(b->gexec, b->stream));
  } else {
    BCK(b, launch_batch_steps(bl, n_steps, b->stream));
  }
  BCK(b, launch_batch_collect(b->d_cases, n, b->d_case_step, b->d_status, b->d_iters, b->d_steps, b->d_iters_sum,
                              b->stream));
  BCK(b, cudaMemcpyAsync(b->h_status, b->d_status, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, b->stream));
  BCK(b, cudaMemcpyAsync(b->h_iters, b->d_iters, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, b->stream));
  BCK(b, cudaMemcpyAsync(b->h_steps, b->d_steps, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, b->stream));
  BCK(b, cudaMemcpyAsync(b->h_iters_sum, b->d_iters_sum, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, b->stream));
  BCK(b, cudaEventRecord(b->done, b->stream));
  b->pending = n_steps;
  return LFM_OK;
}

int lfm_batch_query(lfm_batch* b) {
  if (!b) return bfail(nullptr, LFM_EINVAL, "batch is NULL");
  if (!b->pending) return LFM_OK;
  DeviceGuard g(b->device);
  cudaError_t e = cudaEventQuery(b->done);
  if (e == cudaErrorNotReady) return 1;
  if (e != cudaSuccess) return bfail(b, LFM_ECUDA, "cudaEventQuery: %s", cudaGetErrorString(e));
  return LFM_OK;
}

int lfm_batch_finish(lfm_batch* b) {
  if (!b) return bfail(nullptr, LFM_EINVAL, "batch is NULL");
  if (!b->pending) return LFM_OK;
  DeviceGuard g(b->device);
  b->pending = 0;
  BCK(b, cudaEventSynchronize(b->done));
  int first = LFM_OK;
  for (int i = 0; i < b->n_active; ++i) {
    const int32_t id = b->order[i];
    b->status[id] = b->h_status[i];
    if (b->h_status[i] != 0) {  // a case that stopped early left no seed of its next step to trust
      BCK(b, cudaMemsetAsync(b->slots[id]->cs.flags + 1, 0, sizeof(int32_t), b->stream));
      BCK(b, cudaStreamSynchronize(b->stream));
    }
    b->last_iters[id] = b->h_iters[i];
    b->steps_run[id] = b->h_steps[i];
    b->iters_run[id] = b->h_iters_sum[i];
    if (b->h_iters[i] >= 0) b->est_iters[id] = b->h_iters[i];
    if (b->h_status[i] != 0 && first == LFM_OK) first = b->h_status[i];
  }
  if (first != LFM_OK) return bfail(b, first, "at least one case failed (first status %d)", first);
  if (kCheckedBuild) {
    int site = check_take_batch(b->stream);
    if (site == 0) site = check_take_step(b->stream);
    if (site < 0) return bfail(b, LFM_ECUDA, "reading the index-check word failed");
    if (site > 0) return bfail(b, LFM_EINVAL, "checked build: a kernel met an index out of range (check site %d)", site);
  }
  return LFM_OK;
}

int lfm_batch_case_status(lfm_batch* b, int32_t id) {
  if (!b || id < 0 || id >= (int32_t)b->slots.size()) return LFM_EINVAL;
  return b->status[id];
}

int lfm_batch_case_iters(lfm_batch* b, int32_t id) {
  if (!b || id < 0 || id >= (int32_t)b->slots.size()) return -1;
  return b->last_iters[id];
}

int lfm_batch_results(lfm_batch* b, int32_t* status, int32_t* steps, int32_t* iters, int32_t n) {
  if (!b) return bfail(nullptr, LFM_EINVAL, "batch is NULL");
  if (b->pending) return bfail(b, LFM_ESTATE, "an advance is pending");
  if (n < 0) return bfail(b, LFM_EINVAL, "n = %d is negative", n);
  for (int32_t id = 0; id < n; ++id) {
    const bool live = id < (int32_t)b->slots.size() && b->slots[id] != nullptr;
    if (status) status[id] = live ? b->status[id] : LFM_ESTATE;
    if (steps) steps[id] = live ? b->steps_run[id] : 0;
    if (iters) iters[id] = live ? b->iters_run[id] : 0;
  }
  return LFM_OK;
}

int lfm_batch_case_stats(lfm_batch* b, int32_t id, lfm_step_stats* out, int32_t n) {
  if (!b) return bfail(nullptr, LFM_EINVAL, "batch is NULL");
  if (id < 0 || id >= (int32_t)b->slots.size() || !b->slots[id]) return bfail(b, LFM_EINVAL, "no case %d", id);
  if (b->pending) return bfail(b, LFM_ESTATE, "an advance is pending");
  if (n < 0 || n > kStatsCap) return bfail(b, LFM_EINVAL, "n out of range");
  if (n == 0 || !out) return LFM_OK;
  DeviceGuard g(b->device);
  lfm_ctx* c = b->slots[id];
  BCK(b, cudaMemcpyAsync(out, c->cs.stats, sizeof(lfm_step_stats) * n, cudaMemcpyDeviceToHost, b->stream));
  BCK(b, cudaStreamSynchronize(b->stream));
  return LFM_OK;
}

int lfm_batch_destroy(lfm_batch* b) {
  if (!b) return LFM_OK;
  {
    DeviceGuard g(b->device);
    if (b->pending && b->done) cudaEventSynchronize(b->done);
    for (lfm_ctx* c : b->slots)
      if (c) c->batch = nullptr;
    free_buffers(b);
    if (b->done) cudaEventDestroy(b->done);
    if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
  }
  delete b;
  return LFM_OK;
}

const char* lfm_batch_last_error(const lfm_batch* b) {
  if (b) return b->err.c_str();
  return g_batch_error.c_str();
}

}  // extern "C"

// ---- one case decomposed into parts (the kernels are in lfm_decomp.cu) --------------------

struct lfm_dd {
  lfm_ctx* src = nullptr;             // the configured case whose rows the parts own
  int P = 0;
  int threads = 512;
  int ctas = 0;
  std::string err;
  std::vector<DdPlanPart> plan;
  std::vector<DdPart> parts;          // host copies of the device descriptors
  std::vector<void*> allocs;          // every device allocation, freed by lfm_dd_destroy
  DdPart* d_parts = nullptr;
  int32_t* d_cta_part = nullptr;
  int32_t* d_cta_rank = nullptr;
  SyncWords* sync = nullptr;
  double* partials = nullptr;
  lfm_step_stats* stats = nullptr;
};

namespace {

thread_local std::string g_dd_error;

int ddfail(lfm_dd* d, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (d) d->err = buf;
  g_dd_error = buf;
  return code;
}

#define DDCK(d, call)                                                                       \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) return ddfail(d, LFM_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

template <typename T>
int dd_alloc(lfm_dd* d, T** p, size_t n) {
  void* v = nullptr;
  DDCK(d, cudaMalloc(&v, sizeof(T) * (n > 0 ? n : 1)));
  d->allocs.push_back(v);
  *p = static_cast<T*>(v);
  return LFM_OK;
}

// The decomposed form covers the FP64 step on orthogonal meshes without sources or
// correctors (the benchmark's step).
int dd_case_ok(lfm_dd* d, lfm_ctx* c) {
  if (!c || !c->uploaded) return ddfail(d, LFM_ESTATE, "the case has no mesh uploaded");
  if (c->opts.precision != LFM_FP64) return ddfail(d, LFM_EINVAL, "the decomposed form runs the FP64 step");
  if (c->has_geom || c->n_corr > 0 || c->has_Su || c->has_Sp)
    return ddfail(d, LFM_EINVAL, "the decomposed form covers orthogonal meshes without sources or correctors");
  if (c->pending_steps > 0 || c->batch) return ddfail(d, LFM_ESTATE, "the case is busy (pending advance or batch)");
  return LFM_OK;
}

}  // namespace

extern "C" {

int lfm_dd_plan(int32_t n_cells, int32_t n_faces, const int32_t* owner, const int32_t* neighbour, int32_t n_parts,
                int32_t part, lfm_dd_counts* counts, int32_t* ghost_label, int32_t* send_src, int32_t* send_part,
                int32_t* send_slot) {
  if (n_cells <= 0 || n_faces < 0 || (n_faces > 0 && (!owner || !neighbour)) || !counts)
    return ddfail(nullptr, LFM_EINVAL, "lfm_dd_plan: bad sizes or NULL arrays");
  if (n_parts < 1 || n_parts > n_cells || part < 0 || part >= n_parts)
    return ddfail(nullptr, LFM_EINVAL, "lfm_dd_plan: n_parts must be in [1, n_cells] and part in [0, n_parts)");
  for (int32_t f = 0; f < n_faces; ++f)
    if (owner[f] < 0 || neighbour[f] >= n_cells || neighbour[f] <= owner[f])
      return ddfail(nullptr, LFM_EINVAL, "lfm_dd_plan: face %d out of range or owner >= neighbour", f);
  DdPlanPart pp;
  dd_plan_from_faces(n_cells, n_faces, owner, neighbour, n_parts, part, pp);
  counts->first_label = pp.first;
  counts->n_owned = pp.n_owned;
  counts->n_ghost = (int32_t)pp.ghost.size();
  counts->n_send = (int32_t)pp.send_src.size();
  if (ghost_label) std::copy(pp.ghost.begin(), pp.ghost.end(), ghost_label);
  if (send_src) std::copy(pp.send_src.begin(), pp.send_src.end(), send_src);
  if (send_part) std::copy(pp.send_part.begin(), pp.send_part.end(), send_part);
  if (send_slot) std::copy(pp.send_slot.begin(), pp.send_slot.end(), send_slot);
  return LFM_OK;
}

int lfm_dd_create(lfm_dd** out, lfm_ctx* c, int32_t n_parts) {
  if (!out) return ddfail(nullptr, LFM_EINVAL, "out is NULL");
  *out = nullptr;
  int rc = dd_case_ok(nullptr, c);
  if (rc) return rc;
  if (n_parts < 1 || n_parts > c->N) return ddfail(nullptr, LFM_EINVAL, "n_parts must be in [1, n_cells]");
  DeviceGuard g(c->device);
  const int max_ctas = dd_max_ctas(512, c->W, c->device);
  if (n_parts > max_ctas) return ddfail(nullptr, LFM_EINVAL, "n_parts %d above the %d co-resident CTAs", n_parts, max_ctas);
  lfm_dd* d = new (std::nothrow) lfm_dd;
  if (!d) return ddfail(nullptr, LFM_ENOMEM, "out of host memory");
  d->src = c;
  d->P = n_parts;
  d->ctas = max_ctas;
  auto bail = [&](int code) {
    lfm_dd_destroy(d);
    return code;
  };
  const int32_t N = c->N, W = c->W;
  std::vector<int32_t> slot_other((size_t)W * N);
  if (cudaMemcpyAsync(slot_other.data(), c->cs.slot_other, 4 * (size_t)W * N, cudaMemcpyDeviceToHost, c->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(c->stream) != cudaSuccess)
    return bail(ddfail(nullptr, LFM_ECUDA, "reading the case's addressing failed"));
  d->plan.resize(n_parts);
  d->parts.resize(n_parts);
  // CTAs in proportion to the owned cells, at least one per part
  std::vector<int32_t> share(n_parts, 1);
  {
    int left = max_ctas - n_parts;
    for (int s = 0; s < n_parts; ++s) {
      dd_plan_from_slots(N, W, slot_other.data(), n_parts, s, d->plan[s]);
      const int extra = (int)((int64_t)left * d->plan[s].n_owned / N);
      share[s] += extra;
    }
  }
  std::vector<int32_t> cta_part, cta_rank;
  for (int s = 0; s < n_parts; ++s)
    for (int r = 0; r < share[s]; ++r) {
      cta_part.push_back(s);
      cta_rank.push_back(r);
    }
  d->ctas = (int)cta_part.size();
  for (int s = 0; s < n_parts; ++s) {
    const DdPlanPart& pl = d->plan[s];
    DdPart& pt = d->parts[s];
    pt.N = pl.n_owned;
    pt.G = (int32_t)pl.ghost.size();
    pt.first = pl.first;
    pt.n_send = (int32_t)pl.send_src.size();
    pt.ctas = share[s];
    // local columns: owned label -> label - first, ghost label -> N + its slot, padding -> self
    std::vector<int32_t> loc((size_t)W * pt.N);
    for (int32_t k = 0; k < W; ++k)
      for (int32_t i = 0; i < pt.N; ++i) {
        const int32_t gl = pl.first + i, o = slot_other[(size_t)k * N + gl];
        int32_t v;
        if (o == gl) {
          v = i;
        } else if (o >= pl.first && o < pl.first + pt.N) {
          v = o - pl.first;
        } else {
          const auto it = std::lower_bound(pl.ghost.begin(), pl.ghost.end(), o);
          if (it == pl.ghost.end() || *it != o) return bail(ddfail(nullptr, LFM_ECUDA, "inconsistent ghost list"));
          v = pt.N + (int32_t)(it - pl.ghost.begin());
        }
        loc[(size_t)k * pt.N + i] = v;
      }
    int32_t *sl = nullptr, *ss = nullptr, *sp = nullptr, *sk = nullptr;
    if (dd_alloc(d, &sl, loc.size()) || dd_alloc(d, &ss, pt.n_send) || dd_alloc(d, &sp, pt.n_send) ||
        dd_alloc(d, &sk, pt.n_send) || dd_alloc(d, &pt.x, (size_t)pt.N + pt.G) ||
        dd_alloc(d, &pt.p, (size_t)pt.N + pt.G) || dd_alloc(d, &pt.r, pt.N) || dd_alloc(d, &pt.w, pt.N) ||
        dd_alloc(d, &pt.q, pt.N) || dd_alloc(d, &pt.diag, pt.N) || dd_alloc(d, &pt.rD, pt.N))
      return bail(ddfail(nullptr, LFM_ENOMEM, "device memory for part %d", s));
    pt.slot_local = sl;
    pt.send_src = ss;
    pt.send_part = sp;
    pt.send_slot = sk;
    if (cudaMemcpy(sl, loc.data(), 4 * loc.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        (pt.n_send &&
         (cudaMemcpy(ss, pl.send_src.data(), 4 * (size_t)pt.n_send, cudaMemcpyHostToDevice) != cudaSuccess ||
          cudaMemcpy(sp, pl.send_part.data(), 4 * (size_t)pt.n_send, cudaMemcpyHostToDevice) != cudaSuccess ||
          cudaMemcpy(sk, pl.send_slot.data(), 4 * (size_t)pt.n_send, cudaMemcpyHostToDevice) != cudaSuccess)) ||
        cudaMemcpy(pt.x, c->cs.x + pl.first, 8 * (size_t)pt.N, cudaMemcpyDeviceToDevice) != cudaSuccess ||
        cudaMemset(pt.x + pt.N, 0, 8 * (size_t)(pt.G > 0 ? pt.G : 0)) != cudaSuccess)
      return bail(ddfail(nullptr, LFM_ECUDA, "uploading part %d", s));
  }
  if (dd_alloc(d, &d->d_parts, n_parts) || dd_alloc(d, &d->d_cta_part, cta_part.size()) ||
      dd_alloc(d, &d->d_cta_rank, cta_rank.size()) || dd_alloc(d, &d->sync, 1) ||
      dd_alloc(d, &d->partials, (size_t)kMaxCtas * kMaxSums) || dd_alloc(d, &d->stats, kStatsCap))
    return bail(ddfail(nullptr, LFM_ENOMEM, "device memory for the part table"));
  if (cudaMemcpy(d->d_parts, d->parts.data(), sizeof(DdPart) * n_parts, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(d->d_cta_part, cta_part.data(), 4 * cta_part.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(d->d_cta_rank, cta_rank.data(), 4 * cta_rank.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(d->sync, 0, sizeof(SyncWords)) != cudaSuccess)
    return bail(ddfail(nullptr, LFM_ECUDA, "uploading the part table"));
  *out = d;
  return LFM_OK;
}

int lfm_dd_part_counts(lfm_dd* d, int32_t part, lfm_dd_counts* counts) {
  if (!d || !counts) return ddfail(d, LFM_EINVAL, "NULL argument");
  if (part < 0 || part >= d->P) return ddfail(d, LFM_EINVAL, "part %d out of range", part);
  const DdPart& pt = d->parts[part];
  counts->first_label = pt.first;
  counts->n_owned = pt.N;
  counts->n_ghost = pt.G;
  counts->n_send = pt.n_send;
  return LFM_OK;
}

int lfm_dd_set_field(lfm_dd* d, const double* T) {
  if (!d || !T) return ddfail(d, LFM_EINVAL, "NULL argument");
  DeviceGuard g(d->src->device);
  for (const DdPart& pt : d->parts)
    DDCK(d, cudaMemcpy(pt.x, T + pt.first, 8 * (size_t)pt.N, cudaMemcpyHostToDevice));
  return LFM_OK;
}

int lfm_dd_get_field(lfm_dd* d, double* T) {
  if (!d || !T) return ddfail(d, LFM_EINVAL, "NULL argument");
  DeviceGuard g(d->src->device);
  for (const DdPart& pt : d->parts)
    DDCK(d, cudaMemcpy(T + pt.first, pt.x, 8 * (size_t)pt.N, cudaMemcpyDeviceToHost));
  return LFM_OK;
}

int lfm_dd_advance(lfm_dd* d, int32_t n_steps, lfm_step_stats* out) {
  if (!d) return ddfail(nullptr, LFM_EINVAL, "NULL decomposition");
  if (n_steps < 0 || n_steps > kStatsCap) return ddfail(d, LFM_EINVAL, "n_steps must be in [0, %d]", kStatsCap);
  lfm_ctx* c = d->src;
  int rc = dd_case_ok(d, c);
  if (rc) return rc;
  if (n_steps == 0) return LFM_OK;
  DeviceGuard g(c->device);
  refresh_case(c);
  if ((rc = refresh_coef(c))) return ddfail(d, rc, "coefficient set-up of the case failed");
  CaseDev cs = c->cs;  // the case's rows, with the decomposition's own barrier words and records
  cs.sync = d->sync;
  cs.partials = d->partials;
  cs.stats = d->stats;
  Launch L{d->ctas, d->threads, c->timeout_ns, -1, 0, -1};
  DDCK(d, cudaMemsetAsync(d->sync, 0, sizeof(SyncWords), c->stream));
  DDCK(d, launch_dd_steps(cs, d->d_parts, d->d_cta_part, d->d_cta_rank, L, n_steps, c->stream));
  int32_t status = 0;
  DDCK(d, cudaMemcpyAsync(&status, &d->sync->status, 4, cudaMemcpyDeviceToHost, c->stream));
  std::vector<lfm_step_stats> st(n_steps);
  DDCK(d, cudaMemcpyAsync(st.data(), d->stats, sizeof(lfm_step_stats) * n_steps, cudaMemcpyDeviceToHost, c->stream));
  DDCK(d, cudaStreamSynchronize(c->stream));
  if (out) std::copy(st.begin(), st.end(), out);
  if (status != 0) return ddfail(d, status, "the decomposed step stopped with status %d", status);
  return LFM_OK;
}

int lfm_dd_destroy(lfm_dd* d) {
  if (!d) return LFM_OK;
  {
    DeviceGuard g(d->src ? d->src->device : 0);
    for (void* p : d->allocs) cudaFree(p);
  }
  delete d;
  return LFM_OK;
}

const char* lfm_dd_last_error(const lfm_dd* d) {
  if (d) return d->err.c_str();
  return g_dd_error.c_str();
}

}  // extern "C"

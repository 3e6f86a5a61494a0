// gp_api.cu -- host runtime behind include/gp.h: parameter checks, the physical-units
// nonlinearity, FP64 Crank-Nicolson elimination coefficients and trap tables, the
// device memory layout, TMA descriptors, launch sequencing of the SSCN step, status
// checks and per-sweep event timing.
//
// Paper: program summary ("Solution method": split-step Crank-Nicolson, imaginary
// and real time; "Summary of revisions": physical inputs N, a_s, l_osc turned into
// the dimensionless nonlinearity, energy / chemical potential / rms / integrated
// density outputs, quench by a factor on g, imaginary-to-real-time hand-off).
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/gp.h"
#include "gp_internal.h"

using gpk::FieldParams;
using gpk::SweepParams;

namespace {
thread_local std::string g_create_error = "no error";
}

void gpk::set_thread_error(const char* msg) { g_create_error = msg; }

// Row of the free-line CN operator T_inf = (I + aK)^{-1} (I - aK) (K the second
// difference on the infinite line): the middle row of the zero-ghost operator of a
// line of 2 M + 1 points, M = 64, whose ghosts are so far away (|rho|^64) that their
// influence is far below FP64 rounding for every usable a.  T is symmetric, so that
// row is the Thomas solve (FP64) for the right-hand side (I - aK) e_M.  Returns the
// smallest half-width W in {3, 5, 8} for which the entries beyond distance W sum, in
// modulus, to at most 2^-28 (below FP32 rounding of a result), with
// w[k] = T_inf[M][M + k - W], k = 0 .. 2W; 0 when no such W exists.
int gpk::cn_free_row(std::complex<double> a, std::vector<std::complex<double>>* w) {
  using C = std::complex<double>;
  constexpr int M = 64, n = 2 * M + 1;
  const C b = 1.0 + 2.0 * a;
  std::vector<C> m(n), cp(n), d(n), u(n);
  for (int j = 0; j < n; ++j) {
    m[j] = 1.0 / (j == 0 ? b : b + a * cp[j - 1]);
    cp[j] = -a * m[j];
  }
  C dp = 0.0;
  for (int i = 0; i < n; ++i) {
    const C r = i == M ? 1.0 - 2.0 * a : (i == M - 1 || i == M + 1) ? a : C(0.0);
    dp = (r + a * dp) * m[i];
    d[i] = dp;
  }
  C next = 0.0;
  for (int i = n - 1; i >= 0; --i) next = u[i] = d[i] - cp[i] * next;
  for (int W : {3, 5, gpk::kBandHalfMax}) {
    double tail = 0.0;
    for (int i = 0; i < n; ++i)
      if (std::abs(i - M) > W) tail += std::sqrt(std::norm(u[i]));
    if (!(tail <= std::ldexp(1.0, -28))) continue;
    w->assign(u.begin() + (M - W), u.begin() + (M + W + 1));
    return W;
  }
  return 0;
}

namespace {

constexpr double kPi = 3.14159265358979323846264338327950288;
constexpr size_t kAlign = 256;
constexpr size_t kFastTileBytes = 100 * 1024;   // preferred tile: >= 2 blocks per SM
constexpr size_t kMaxTileBytes = 226 * 1024;    // opt-in shared memory per block, minus slack
constexpr int kBandMinNx = 8;                   // one reflection covers every window
constexpr int kBandStages = 3;                  // rows in flight per warp of the x band kernel
constexpr size_t kBandBlockBytes = 100 * 1024;  // above this, 2 stages
constexpr size_t kBandWarpBudget = 6 * 1024;   // x band: row slots of one warp for groups of rows

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Geometry of one sweep in one mode (0: real field, 1: complex field).
struct SweepGeom {
  int lines = 0;      // lines per tile
  int box = 0;        // TMA box length along the line (y / z) -- x: unused
  int nbox = 0;
  size_t smem = 0;    // dynamic shared memory bytes of one block
};

struct Layout {
  size_t rbytes = 8;               // bytes of one real value (8 FP64, 4 FP32)
  int pitch[2] = {0, 0};           // row pitch in elements, per mode
  size_t field_bytes = 0;
  size_t off_field = 0, off_staging = 0, off_coef = 0, off_vtab = 0, off_otab = 0;
  size_t off_partials = 0, off_scalars = 0, total = 0;
  size_t coef_off[2][3][2] = {};   // [mode][axis][A/B] byte offset from off_coef
  size_t fx_off[2] = {};           // trap factors along x per mode [pitch], from off_coef
  size_t fyz_off[2] = {};          // trap factor per row per mode, from off_coef
  size_t fxh_off[2] = {};          // the same for half a step (Strang splitting)
  size_t fyzh_off[2] = {};
  size_t npartials = 0;
  SweepGeom geom[2][3];
  long long ntiles_z[2] = {0, 0};
  int tiles_x[2][3] = {};
};

// Largest power-of-two line count (<= 32) whose tile fits `budget`; for TMA tiles the
// tile's inner extent must be a multiple of 16 bytes.
int choose_lines(size_t line_bytes, size_t elem_bytes, bool tma_inner, size_t budget) {
  for (int w = 32; w >= 1; w >>= 1) {
    if (tma_inner && ((size_t)w * elem_bytes) % 16 != 0) return 0;
    if ((size_t)w * line_bytes + 64 <= budget) return w;
  }
  return 0;
}

const char* check_params(const gp_params* p) {
  if (!p) return "params is NULL";
  const int n[3] = {p->nx, p->ny, p->nz};
  for (int a = 0; a < 3; ++a)
    if ((n[a] < 3 && !(a == 2 && n[a] == 1)) || n[a] > gpk::kMaxExtent)
      return "grid extents must be within 3..2048 (nz = 1: a 2D solve)";
  const double h[3] = {p->dx, p->dy, p->dz};
  for (int a = 0; a < 3; ++a)
    if (!(h[a] > 0.0) || !std::isfinite(h[a])) return "grid spacings must be finite and > 0";
  if (!(p->dt > 0.0) || !std::isfinite(p->dt)) return "dt must be finite and > 0";
  if (!(p->gamma > 0.0) || !(p->nu > 0.0) || !(p->lambda > 0.0) || !std::isfinite(p->gamma) ||
      !std::isfinite(p->nu) || !std::isfinite(p->lambda))
    return "trap ratios gamma, nu, lambda must be finite and > 0";
  if (p->use_physical != 0 && p->use_physical != 1) return "use_physical must be 0 or 1";
  if (p->use_physical) {
    if (!std::isfinite(p->natoms) || !std::isfinite(p->a_s) || !(p->l_osc > 0.0) ||
        !std::isfinite(p->l_osc))
      return "physical inputs need finite natoms, a_s and l_osc > 0";
  } else if (!std::isfinite(p->g)) {
    return "g must be finite";
  }
  if (p->prec != GP_F64 && p->prec != GP_F32) return "prec must be GP_F64 or GP_F32";
  return nullptr;
}

// g = 4 pi N a_s / l_osc, or g as given.
double nonlinearity(const gp_params* p) {
  return p->use_physical ? 4.0 * kPi * p->natoms * p->a_s / p->l_osc : p->g;
}

const char* compute_layout(const gp_params* p, Layout* L) {
  L->rbytes = p->prec == GP_F64 ? 8 : 4;
  const int n[3] = {p->nx, p->ny, p->nz};
  const size_t N = (size_t)p->nx * p->ny * p->nz;
  for (int m = 0; m < 2; ++m) {
    const size_t eb = L->rbytes * (m + 1);          // element bytes
    const size_t q = 16 / eb > 0 ? 16 / eb : 1;     // pitch multiple: rows start 16-byte aligned
    L->pitch[m] = (int)align_up((size_t)p->nx, q);
  }
  const size_t rows = (size_t)p->ny * p->nz;
  L->field_bytes = std::max((size_t)L->pitch[0] * L->rbytes, (size_t)L->pitch[1] * 2 * L->rbytes) * rows;

  for (int m = 0; m < 2; ++m) {
    const size_t eb = L->rbytes * (m + 1);
    // x sweep: tile = lines x pitch, contiguous
    {
      const size_t line = (size_t)L->pitch[m] * eb;
      int w = choose_lines(line, eb, false, kFastTileBytes);
      if (!w) w = choose_lines(line, eb, false, kMaxTileBytes);
      if (!w) return "x extent too large for one shared-memory row tile";
      L->geom[m][0].lines = w;
      L->geom[m][0].smem = (size_t)w * line + 64;
    }
    for (int a = 1; a < 3; ++a) {
      SweepGeom& G = L->geom[m][a];
      G.nbox = (n[a] + gpk::kMaxBox - 1) / gpk::kMaxBox;
      G.box = (n[a] + G.nbox - 1) / G.nbox;
      const size_t line = (size_t)G.nbox * G.box * eb;
      int w = choose_lines(line, eb, true, kFastTileBytes);
      if (!w) w = choose_lines(line, eb, true, kMaxTileBytes);
      if (!w) return "line too long for one shared-memory tile";
      G.lines = w;
      G.smem = (size_t)w * line + 64;
      L->tiles_x[m][a] = (p->nx + w - 1) / w;
    }
    L->ntiles_z[m] = (long long)L->tiles_x[m][2] * p->ny;
  }

  size_t off = 0;
  L->off_field = off;
  off = align_up(off + L->field_bytes, kAlign);
  L->off_staging = off;
  off = align_up(off + N * 16, kAlign);
  L->off_coef = off;
  size_t c = 0;
  for (int m = 0; m < 2; ++m)
    for (int a = 0; a < 3; ++a)
      for (int ab = 0; ab < 2; ++ab) {
        L->coef_off[m][a][ab] = c;
        c = align_up(c + (size_t)n[a] * L->rbytes * (m + 1), kAlign);
      }
  for (int m = 0; m < 2; ++m)
    for (int half = 0; half < 2; ++half) {
      (half ? L->fxh_off : L->fx_off)[m] = c;
      c = align_up(c + (size_t)L->pitch[m] * L->rbytes * (m + 1), kAlign);
      (half ? L->fyzh_off : L->fyz_off)[m] = c;
      c = align_up(c + rows * L->rbytes * (m + 1), kAlign);
    }
  off = align_up(off + c, kAlign);
  L->off_vtab = off;
  off = align_up(off + (size_t)(p->nx + p->ny + p->nz) * L->rbytes, kAlign);
  L->off_otab = off;
  off = align_up(off + (size_t)2 * (p->nx + p->ny + p->nz) * 8, kAlign);
  L->off_partials = off;
  L->npartials = std::max<size_t>((size_t)std::max(L->ntiles_z[0], L->ntiles_z[1]),
                                  (size_t)gpk::kReduceBlocks * gpk::kObsAcc);
  off = align_up(off + L->npartials * 8, kAlign);
  L->off_scalars = off;
  off = align_up(off + 512, kAlign);
  L->total = off;
  return nullptr;
}

// Thomas pivots of (1+2a) u_j - a (u_{j-1}+u_{j+1}): m_0 = 1/b, m_j = 1/(b - a^2 m_{j-1}),
// b = 1 + 2a (so that cp_j = -a m_j); the sweeps use A_j = m_j (1-2a), B_j = a m_j.
void cn_coefficients(int n, std::complex<double> a, std::vector<std::complex<double>>* A,
                     std::vector<std::complex<double>>* B) {
  const std::complex<double> b = 1.0 + 2.0 * a;
  A->resize(n);
  B->resize(n);
  std::complex<double> cp_prev = 0.0;
  for (int j = 0; j < n; ++j) {
    const std::complex<double> m = 1.0 / (j == 0 ? b : b + a * cp_prev);
    cp_prev = -a * m;
    (*A)[j] = m * (1.0 - 2.0 * a);
    (*B)[j] = a * m;
  }
}

// GP_SWEEP_KERNELS=tile makes every sweep use the shared-memory tile kernels;
// GP_SWEEP_KERNELS=stream keeps the FP32 sweeps on the streaming recurrence kernels
// instead of the banded ones (stream_x: only x, stream_yz: only y and z); for
// diagnostics and A/B measurements.  Any other value or none: automatic choice.
bool force_tile() {
  const char* v = std::getenv("GP_SWEEP_KERNELS");
  return v && std::strcmp(v, "tile") == 0;
}
// GP_NORM_DEFER=0 makes the FP32 banded z sweep finish its norm itself (last block)
// instead of leaving the sum of its partials to the next x sweep (A/B measurements).
bool norm_defer_enabled() {
  const char* v = std::getenv("GP_NORM_DEFER");
  return !(v && std::strcmp(v, "0") == 0);
}
// GP_X_REG=0 keeps the banded x sweep on the copy-fed kernel for rows that the
// register-row kernel could take (A/B measurements).
bool x_reg_enabled() {
  const char* v = std::getenv("GP_X_REG");
  return !(v && std::strcmp(v, "0") == 0);
}
// GP_BAND_PREFETCH=0 keeps the banded y / z sweeps' turn loads in registers instead
// of copying them to shared memory one turn ahead (A/B measurements).
// GP_BAND_SEG_TURNS=k fixes the banded y / z segments at k turns of 2W+1 points
// instead of the occupancy model's choice (A/B measurements).
int band_seg_turns() {
  const char* v = std::getenv("GP_BAND_SEG_TURNS");
  return v ? std::max(0, std::atoi(v)) : 0;
}
bool band_prefetch() {
  const char* v = std::getenv("GP_BAND_PREFETCH");
  return !(v && std::strcmp(v, "0") == 0);
}
bool force_stream() {
  const char* v = std::getenv("GP_SWEEP_KERNELS");
  return v && (std::strcmp(v, "stream") == 0 || std::strcmp(v, "stream_x") == 0);
}
bool force_stream_yz() {
  const char* v = std::getenv("GP_SWEEP_KERNELS");
  return v && (std::strcmp(v, "stream") == 0 || std::strcmp(v, "stream_yz") == 0);
}


PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
  }
  return fn;
}

struct TimedLaunch {
  cudaEvent_t start, stop;
  int axis;
};

}  // namespace

struct gp_solver {
  gp_params prm;
  Layout L;
  double g = 0.0;
  int device = 0;
  cudaStream_t stream = nullptr;
  bool owns = false;
  unsigned char* base = nullptr;
  bool is_complex = false;
  // device pointers
  void* field = nullptr;
  double* staging = nullptr;
  void* vtab = nullptr;
  double* otab = nullptr;
  double* partials = nullptr;
  double* scale = nullptr;
  int* status = nullptr;
  unsigned int* counters = nullptr;  // [0] sweeps, [1] reductions
  double* obs = nullptr;
  SweepParams sp[2][3];
  int head[2][3] = {};               // see SweepParams::head
  int trunc[2][3] = {};              // FP32 fast sweeps: truncation depth, 0 = use the tile kernel
  int fast_grid[2][3] = {};          // blocks of the fast sweeps (x band: persistent grid)
  int band_w[2][3] = {};             // FP32 banded sweep half-width per mode and axis, 0 = not used
  bool line64 = false;               // FP64 field: the line-streaming sweeps of gp_sweeps64.cu
  bool defer_norm = false;           // FP32 real field: the z sweep's norm finished by its reader
  int* scale_state = nullptr;        // device: 1 while the factor is in the z sweep's partials
  unsigned int* step_ctr = nullptr;  // device: imaginary-time steps since the field was set
                                     // (the FP32 factor's dither, step_dither)
  int split = GP_SPLIT_LIE;          // splitting of a step
  bool kinetic_only = false;         // x sweep without the pointwise substep (Strang)
  float band_wt[2][3][2 * 17] = {};  // its weights (complex: pairs)
  int nsm = 0;
  CUtensorMap tmap[2][3];  // [mode][axis]; axis 0 unused (64-byte aligned type)
  // one Lie / Strang step as a CUDA graph per mode, captured on first use on cap_stream
  cudaGraphExec_t step_exec[2] = {nullptr, nullptr};
  cudaGraphExec_t strang_exec[2] = {nullptr, nullptr};
  cudaStream_t cap_stream = nullptr;
  // overlapped field reads (gp_get_psi_f32_async): the field is packed into one of the
  // two halves of export_buf (allocated on first use, the halves taken in turn) and
  // copied to host on copy_stream; a packing into a half waits for that half's previous
  // copy (copy_done[half]), the host-completing calls for both
  void* export_buf = nullptr;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t copy_ready = nullptr, copy_done[2] = {nullptr, nullptr};
  bool copy_pending[2] = {false, false};
  int export_next = 0;
  // overlapped field writes (gp_set_psi_f32_async): the host field is copied into
  // one of the two halves of put_buf (allocated on first use, the halves taken in turn)
  // on put_stream; the next call that touches the field waits for put_ready, moves the
  // half into the field on the solver stream and records that half's put_free, which
  // the write after next waits for before it reuses the half
  void* put_buf = nullptr;
  cudaStream_t put_stream = nullptr;
  cudaEvent_t put_ready = nullptr, put_free[2] = {nullptr, nullptr};
  bool put_pending = false, put_complex = false;
  int put_half = 0, put_next = 0;
  bool step_graph = true;            // false once capture failed: direct launches only
  // timing
  bool timing = false;
  std::vector<TimedLaunch> pending;
  std::vector<cudaEvent_t> pool;
  std::string err = "no error";
};

namespace {

int fail(gp_solver* s, int code, const std::string& msg) {
  if (s) s->err = msg;
  return code;
}

int cuda_fail(gp_solver* s, cudaError_t e, const char* where) {
  return fail(s, GP_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define GP_CUDA(s, call)                                   \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail((s), e_, #call); \
  } while (0)

// The factor of a solver whose z sweep defers its norm: sum the partials into it when
// they are newer than it (one small kernel on the solver's stream; nothing otherwise).
void resolve_scale(gp_solver* s) {
  if (!s->defer_norm) return;
  const cudaError_t e =
      gpk::launch_resolve_scale(s->scale, s->scale_state, s->partials,
                                (int)s->fast_grid[0][2], s->prm.dx * s->prm.dy * s->prm.dz,
                                s->status, s->stream);
  if (e != cudaSuccess) cuda_fail(s, e, "resolve scale");
}

// Arguments of the reductions, I/O and pointwise kernels, which all read the pending
// factor: a deferred one is resolved first.
FieldParams field_params(gp_solver* s) {
  resolve_scale(s);
  FieldParams f;
  f.psi = s->field;
  f.nx = s->prm.nx;
  f.ny = s->prm.ny;
  f.nz = s->prm.nz;
  f.pitch = s->L.pitch[s->is_complex ? 1 : 0];
  f.scale = s->scale;
  f.partials = s->partials;
  f.counter = s->counters + 1;
  f.out = s->obs;
  f.status = s->status;
  f.tab = s->otab;
  f.hx = s->prm.dx;
  f.hy = s->prm.dy;
  f.hz = s->prm.nz == 1 ? 1.0 : s->prm.dz;   // 2D: cell area hx hy
  f.g = s->g;
  return f;
}

int encode_maps(gp_solver* s) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return fail(s, GP_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
  const gp_params& p = s->prm;
  for (int m = 0; m < 2; ++m) {
    const int wpe = m + 1;
    const size_t eb = s->L.rbytes * wpe;
    const CUtensorMapDataType dt =
        s->L.rbytes == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    const cuuint64_t dims[3] = {(cuuint64_t)p.nx * wpe, (cuuint64_t)p.ny, (cuuint64_t)p.nz};
    const cuuint64_t strides[2] = {(cuuint64_t)s->L.pitch[m] * eb,
                                   (cuuint64_t)s->L.pitch[m] * eb * p.ny};
    const cuuint32_t estr[3] = {1, 1, 1};
    for (int a = 1; a < 3; ++a) {
      const SweepGeom& G = s->L.geom[m][a];
      const cuuint32_t box[3] = {(cuuint32_t)(G.lines * wpe), a == 1 ? (cuuint32_t)G.box : 1u,
                                 a == 2 ? (cuuint32_t)G.box : 1u};
      CUresult r = enc(&s->tmap[m][a], dt, 3, s->field, dims, strides, box, estr,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                       CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) {
        char buf[128];
        snprintf(buf, sizeof buf, "cuTensorMapEncodeTiled failed (%d) for mode %d axis %d", (int)r,
                 m, a);
        return fail(s, GP_ERR_CUDA, buf);
      }
    }
  }
  return GP_OK;
}

void fill_sweep_params(gp_solver* s) {
  const gp_params& p = s->prm;
  const int n[3] = {p.nx, p.ny, p.nz};
  unsigned char* coef = s->base + s->L.off_coef;
  const size_t rb = s->L.rbytes;
  unsigned char* vt = static_cast<unsigned char*>(s->vtab);
  for (int m = 0; m < 2; ++m)
    for (int a = 0; a < 3; ++a) {
      SweepParams& q = s->sp[m][a];
      std::memset(&q, 0, sizeof q);
      q.psi = s->field;
      q.out = s->field;
      q.nx = p.nx;
      q.ny = p.ny;
      q.nz = p.nz;
      q.pitch = s->L.pitch[m];
      q.n = n[a];
      q.lines = s->L.geom[m][a].lines;
      q.tiles_x = s->L.tiles_x[m][a];
      q.box = s->L.geom[m][a].box;
      q.nbox = s->L.geom[m][a].nbox;
      q.words_per_elem = m + 1;
      q.A = coef + s->L.coef_off[m][a][0];
      q.B = coef + s->L.coef_off[m][a][1];
      q.head = s->head[m][a];
      q.vx = vt;
      q.vy = vt + (size_t)p.nx * rb;
      q.vz = vt + (size_t)(p.nx + p.ny) * rb;
      q.dt = p.dt;
      q.g = s->g;
      q.band_dtg = (float)(p.dt * s->g);
      q.pw = 1;
      q.scale = s->scale;
      // FP32 field in imaginary time: the renormalisation factor is dithered per step
      q.step_ctr = (m == 0 && s->L.rbytes == 4) ? s->step_ctr : nullptr;
      q.partials = s->partials;
      q.counter = s->counters;
      q.scale_out = s->scale;
      q.status = s->status;
      q.wait_ns = gpk::kWaitLimitNs;
      q.dV = p.dx * p.dy * p.dz;
      q.ntiles = s->L.ntiles_z[m];
      q.trunc = s->trunc[m][a];
      if (q.trunc) {
        const int tiles32 = (p.nx + 31) / 32;
        q.tiles_x = tiles32;
        const long long rows = (long long)p.ny * p.nz;
        long long warps = rows;
        if (a > 0) {
          // split lines into segments: choose the count that best fills whole waves of
          // resident warps, charging each segment its 2L+1 elements of warm-up;
          // segments stay >= 4 (L+1) long
          const long long lines = (long long)tiles32 * (a == 1 ? p.nz : p.ny);
          const long long cap =
              (long long)s->nsm * gpk::stream_warps_per_sm(a, m == 1, q.trunc);
          const int nmax = std::max(1, n[a] / (4 * (q.trunc + 1)));
          int nseg = 1;
          double best = 0.0;
          for (int c = 1; c <= nmax; ++c) {
            const long long items = lines * c;
            const long long waves = (items + cap - 1) / cap;
            const double fill = (double)items / (double)(waves * cap);
            const int seglen = (n[a] + c - 1) / c;
            const double work = (double)(seglen + (c > 1 ? 2 * q.trunc + 1 : q.trunc)) / seglen;
            const double eff = fill / work;
            if (eff > best * 1.02) {
              best = eff;
              nseg = c;
            }
          }
          // one FP64 norm partial per block must fit the partials area
          while (nseg > 1 && (lines * nseg + 3) / 4 > (long long)s->L.npartials) --nseg;
          q.nseg = nseg;
          warps = lines * q.nseg;
          q.psi = a == 1 ? (void*)s->field : (void*)s->staging;
          q.out = a == 1 ? (void*)s->staging : (void*)s->field;
        }
        long long blocks = (warps + 3) / 4;   // x: capped at the resident grid by the launcher
        s->fast_grid[m][a] = (int)blocks;
      }
      q.band_fx = coef + s->L.fx_off[m];
      q.band_fyz = coef + s->L.fyz_off[m];
      if (a == 0 && s->band_w[m][0]) {
        std::memcpy(q.band_wt, s->band_wt[m][0], sizeof q.band_wt);
        q.band_w = s->band_w[m][0];
        const size_t slot_bytes = ((size_t)s->L.pitch[m] + 16) * rb * (m + 1);
        q.band_stages = gpk::kBandWarps * kBandStages * slot_bytes <= kBandBlockBytes ? kBandStages : 2;
        // rows of 32 or more 16-byte vectors fill the lanes one at a time; shorter
        // rows are taken in groups
        const int ept = m == 0 ? 4 : 2;
        q.band_group = (p.nx + ept - 1) / ept >= 32
                           ? 1
                           : gpk::x_band_group(p.nx, ept, q.band_stages, slot_bytes, kBandWarpBudget);
        const size_t smem = gpk::x_band_smem(q, m == 1);
        int bps = 0;
        if (gpk::x_band_prepare(q.band_w, m == 1, q.band_group > 1, smem, &bps) == cudaSuccess &&
            bps > 0) {
          // rows per warp such that every warp is resident at once with equal work
          const long long rows = (long long)p.ny * p.nz;
          const long long warps = std::min((long long)s->nsm * bps * gpk::kBandWarps, rows);
          q.band_rows = (int)(rows / warps);
          q.band_rem = (int)(rows % warps);
          s->fast_grid[m][0] = (int)((warps + gpk::kBandWarps - 1) / gpk::kBandWarps);
        } else {
          cudaGetLastError();
          s->band_w[m][0] = 0;
          q.band_w = 0;
        }
        // real rows of nx = 8 m <= 256 points: the row in registers, no copies (complex
        // rows measured no faster that way)
        int rbps = 0;
        if (q.band_w && m == 0 && gpk::x_reg_fits(p.nx, q.band_w) && x_reg_enabled() &&
            gpk::x_reg_prepare(q.band_w, m == 1, &rbps) == cudaSuccess && rbps > 0) {
          const long long rows = (long long)p.ny * p.nz;
          const long long warps = std::min((long long)s->nsm * rbps * gpk::kXRegWarps, rows);
          q.band_rows = (int)(rows / warps);
          q.band_rem = (int)(rows % warps);
          s->fast_grid[m][0] = (int)((warps + gpk::kXRegWarps - 1) / gpk::kXRegWarps);
          q.band_reg = 1;
        }
        cudaGetLastError();
      }
      if (a > 0 && s->band_w[m][a]) {
        std::memcpy(q.band_wt, s->band_wt[m][a], sizeof q.band_wt);
        q.band_w = s->band_w[m][a];
        q.psi = a == 1 ? (void*)s->field : (void*)s->staging;
        q.out = a == 1 ? (void*)s->staging : (void*)s->field;
        // segment length: the fewest whole turns of the ring (2W+1 points) that make at
        // least 10 points.  Measured on GB300 (graph-replayed steps): at W = 5, 11-point
        // segments (two waves of resident threads) beat the 22-point ones a fill model
        // chose (one wave) by 2.3 us per 240x200x160 step and by 2 % at 512x400x320; at
        // W = 3 (real time), 14 points ran 66.2 us per step against 71.8 us at 7 (six
        // halo loads per seven outputs) and 66.7 us with the fill model's choice
        const int P = 2 * q.band_w + 1;
        const int ept = m == 0 ? 4 : 2;
        const long long cols = (long long)((p.nx + ept - 1) / ept) * (a == 1 ? p.nz : p.ny);
        q.band_cp = band_prefetch() ? 1 : 0;
        // (sets the kernel's shared-memory limit, above 48 KB at W = 8)
        gpk::band_line_blocks_per_sm(a, m == 1, q.band_w, q.band_cp != 0);
        const int forced = band_seg_turns();
        int best_seg = std::min((forced > 0 ? forced : (10 + P - 1) / P) * P, std::max(n[a], P));
        // one FP64 norm partial per block must fit the partials area
        long long blocks = 0;
        for (;; best_seg += P) {
          blocks = (cols * ((n[a] + best_seg - 1) / best_seg) + 127) / 128;
          if (blocks <= (long long)s->L.npartials || best_seg >= n[a]) break;
        }
        q.band_seg = best_seg;
        s->fast_grid[m][a] = (int)blocks;
      }
    }
  // FP32 real field, banded x and z sweeps: the z sweep only stores its norm partials
  // and the next x sweep sums them (every block, in the same order) into the factor it
  // applies, instead of the last z block summing them at the end of the z sweep; other
  // readers of the factor resolve it first (resolve_scale)
  s->defer_norm = s->L.rbytes == 4 && p.nz > 1 && s->band_w[0][0] && s->band_w[0][2] &&
                  norm_defer_enabled();
  for (int a = 0; a < 3; ++a) {
    SweepParams& q = s->sp[0][a];
    q.norm_defer = s->defer_norm && a != 1 ? 1 : 0;
    q.norm_blocks = s->fast_grid[0][2];
    q.norm_copies = std::max(1, std::min(8, (int)(s->L.npartials / std::max(1, s->fast_grid[0][2]))));
    q.scale_state = s->scale_state;
  }
}

template <class T> void put(std::vector<unsigned char>& buf, size_t off, const T& v) {
  std::memcpy(buf.data() + off, &v, sizeof(T));
}

// Host tables (coefficients in the storage precision, trap tables), one upload.
int upload_tables(gp_solver* s) {
  const gp_params& p = s->prm;
  const Layout& L = s->L;
  const int n[3] = {p.nx, p.ny, p.nz};
  const double h[3] = {p.dx, p.dy, p.dz};
  const double w[3] = {p.gamma, p.nu, p.lambda};
  const bool f64 = L.rbytes == 8;
  const size_t span = L.off_partials - L.off_coef;
  std::vector<unsigned char> buf(span, 0);
  auto put_real = [&](size_t off, double v) {
    if (f64) put<double>(buf, off, v);
    else put<float>(buf, off, (float)v);
  };
  for (int m = 0; m < 2; ++m)
    for (int a = 0; a < 3; ++a) {
      const double beta = p.dt / (4.0 * h[a] * h[a]);
      const std::complex<double> alpha = m == 0 ? std::complex<double>(beta, 0.0)
                                                : std::complex<double>(0.0, beta);
      std::vector<std::complex<double>> A, B;
      cn_coefficients(n[a], alpha, &A, &B);
      // first index from which every coefficient, rounded to the storage precision,
      // equals the last one: the kernels keep that value in registers
      auto rounded = [&](std::complex<double> c) {
        return f64 ? c : std::complex<double>((float)c.real(), (float)c.imag());
      };
      int head = n[a];
      while (head > 0 && rounded(A[head - 1]) == rounded(A[n[a] - 1]) &&
             rounded(B[head - 1]) == rounded(B[n[a] - 1]))
        --head;
      s->head[m][a] = head;
      // FP32: the coupling beyond distance L, |B|^L, must stay below 2^-30
      s->trunc[m][a] = 0;
      if (!f64 && head <= 8 && !force_tile()) {
        const double bmag = std::abs(rounded(B[n[a] - 1]));
        for (int depth : {3, 5, 8})
          if (std::pow(bmag, depth + 1) <= std::ldexp(1.0, -30)) {
            s->trunc[m][a] = depth;
            break;
          }
        // x: the streaming kernel needs head <= 32 - L (chunk geometry): always true here
      }
      for (int ab = 0; ab < 2; ++ab) {
        const std::vector<std::complex<double>>& C = ab == 0 ? A : B;
        size_t off = L.coef_off[m][a][ab];
        for (int j = 0; j < n[a]; ++j) {
          if (m == 0) {
            put_real(off + j * L.rbytes, C[j].real());
          } else {
            put_real(off + 2 * j * L.rbytes, C[j].real());
            put_real(off + (2 * j + 1) * L.rbytes, C[j].imag());
          }
        }
      }
    }
  // FP32 sweeps as banded operators on the odd extension of each line, when a
  // half-width <= 8 is exact to FP32 rounding and the line has >= kBandMinNx points
  for (int m = 0; m < 2; ++m)
    for (int a = 0; a < 3; ++a) {
      s->band_w[m][a] = 0;
      if (f64 || force_tile() || n[a] < kBandMinNx) continue;
      if (force_stream() && a == 0) continue;
      if (force_stream_yz() && a > 0) continue;
      const double beta = p.dt / (4.0 * h[a] * h[a]);
      std::vector<std::complex<double>> w;
      const int W = gpk::cn_free_row(m == 0 ? std::complex<double>(beta, 0.0)
                                       : std::complex<double>(0.0, beta), &w);
      if (!W) continue;
      s->band_w[m][a] = W;
      w[W] -= 1.0;   // the kernels add the identity part separately
      for (int k = 0; k <= 2 * W; ++k) {
        if (m == 0) {
          s->band_wt[m][a][k] = (float)w[k].real();
        } else {
          s->band_wt[m][a][2 * k] = (float)w[k].real();
          s->band_wt[m][a][2 * k + 1] = (float)w[k].imag();
        }
      }
    }
  // 2D (nz = 1): no z sweep; a fast (out-of-place) y sweep is followed by a copy of
  // the staging area back to the field
  if (p.nz == 1)
    for (int m = 0; m < 2; ++m) s->trunc[m][2] = s->band_w[m][2] = 0;
  // the FP32 y / z kernels (banded or streaming) write out of place (y: field ->
  // staging, z: staging -> field), so in 3D they are used together or not at all
  for (int m = 0; m < 2 && p.nz > 1; ++m)
    if (!(s->trunc[m][1] || s->band_w[m][1]) || !(s->trunc[m][2] || s->band_w[m][2])) {
      s->trunc[m][1] = s->trunc[m][2] = 0;
      s->band_w[m][1] = s->band_w[m][2] = 0;
    }
  // potential tables V_a(x) = w_a^2 x^2 / 2 in storage precision, and FP64 copies + x^2
  const size_t vt = L.off_vtab - L.off_coef, ot = L.off_otab - L.off_coef;
  size_t iv = 0;
  const int ntot = p.nx + p.ny + p.nz;
  for (int a = 0; a < 3; ++a)
    for (int i = 0; i < n[a]; ++i, ++iv) {
      const double x = (i - 0.5 * (n[a] - 1)) * h[a];
      const double V = 0.5 * w[a] * w[a] * x * x;
      put_real(vt + iv * L.rbytes, V);
      put<double>(buf, ot + iv * 8, V);
      put<double>(buf, ot + (ntot + iv) * 8, x * x);
    }
  // trap factors of the pointwise substep, exp(-dt V) (real field) and
  // cis(-dt V) = (cos dt V, -sin dt V) (complex field), separable as a factor along x
  // and one per row; computed in FP64, rounded once to the storage precision
  {
    const size_t rb = L.rbytes;
    auto pot = [&](int a, int i) {
      const double x = (i - 0.5 * (n[a] - 1)) * h[a];
      return 0.5 * w[a] * w[a] * x * x;
    };
    for (int half = 0; half < 2; ++half) {
      const double tau = half ? 0.5 * p.dt : p.dt;
      const size_t* fxo = half ? L.fxh_off : L.fx_off;
      const size_t* fyo = half ? L.fyzh_off : L.fyz_off;
      for (int i = 0; i < p.nx; ++i) {
        const double th = tau * pot(0, i);
        put_real(fxo[0] + (size_t)i * rb, std::exp(-th));
        put_real(fxo[1] + (size_t)i * 2 * rb, std::cos(th));
        put_real(fxo[1] + (size_t)i * 2 * rb + rb, -std::sin(th));
      }
      for (int k = 0; k < p.nz; ++k)
        for (int j = 0; j < p.ny; ++j) {
          const double th = tau * (pot(1, j) + pot(2, k));
          const size_t r = (size_t)k * p.ny + j;
          put_real(fyo[0] + r * rb, std::exp(-th));
          put_real(fyo[1] + r * 2 * rb, std::cos(th));
          put_real(fyo[1] + r * 2 * rb + rb, -std::sin(th));
        }
    }
  }
  GP_CUDA(s, cudaMemcpyAsync(s->base + L.off_coef, buf.data(), span, cudaMemcpyHostToDevice,
                             s->stream));
  GP_CUDA(s, cudaStreamSynchronize(s->stream));
  return GP_OK;
}

__global__ void k_set_scale_one(double* scale, int* state) {
  *scale = 1.0;
  *state = 0;
}

int set_scale_one(gp_solver* s) {
  k_set_scale_one<<<1, 1, 0, s->stream>>>(s->scale, s->scale_state);
  GP_CUDA(s, cudaGetLastError());
  return GP_OK;
}

// A new field: its imaginary-time steps (the FP32 factor's dither) count from zero, so
// that the same field and the same steps give the same bits in any solver.
int reset_steps(gp_solver* s) {
  GP_CUDA(s, cudaMemsetAsync(s->step_ctr, 0, sizeof(unsigned int), s->stream));
  return GP_OK;
}

int create_impl(const gp_params* p, void* dev_buf, size_t bytes, void* stream, gp_solver** out) {
  if (!out) {
    g_create_error = "out is NULL";
    return GP_ERR_ARG;
  }
  *out = nullptr;
  if (const char* why = check_params(p)) {
    g_create_error = why;
    return GP_ERR_ARG;
  }
  gp_solver* s = new gp_solver();
  s->prm = *p;
  if (const char* why = compute_layout(p, &s->L)) {
    g_create_error = why;
    delete s;
    return GP_ERR_ARG;
  }
  s->g = nonlinearity(p);
  s->stream = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaGetDevice(&s->device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&s->nsm, cudaDevAttrMultiProcessorCount, s->device);
  if (e != cudaSuccess) {
    g_create_error = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
    delete s;
    return GP_ERR_CUDA;
  }
  if (dev_buf) {
    if (bytes < s->L.total || (reinterpret_cast<uintptr_t>(dev_buf) % kAlign) != 0) {
      g_create_error = "caller buffer too small or not 256-byte aligned";
      delete s;
      return GP_ERR_NOMEM;
    }
    s->base = static_cast<unsigned char*>(dev_buf);
  } else {
    e = cudaMalloc(&s->base, s->L.total);
    if (e != cudaSuccess) {
      cudaGetLastError();
      g_create_error = std::string("cudaMalloc: ") + cudaGetErrorString(e);
      delete s;
      return GP_ERR_NOMEM;
    }
    s->owns = true;
  }
  const Layout& L = s->L;
  s->field = s->base + L.off_field;
  s->staging = reinterpret_cast<double*>(s->base + L.off_staging);
  s->vtab = s->base + L.off_vtab;
  s->otab = reinterpret_cast<double*>(s->base + L.off_otab);
  s->partials = reinterpret_cast<double*>(s->base + L.off_partials);
  unsigned char* sc = s->base + L.off_scalars;
  s->scale = reinterpret_cast<double*>(sc);
  s->obs = reinterpret_cast<double*>(sc + 64);
  s->status = reinterpret_cast<int*>(sc + 256);
  s->scale_state = reinterpret_cast<int*>(sc + 160);
  s->step_ctr = reinterpret_cast<unsigned int*>(sc + 192);
  s->counters = reinterpret_cast<unsigned int*>(sc + 320);

  int rc = GP_OK;
  auto bail = [&](int code) {
    g_create_error = s->err;
    gp_destroy(s);
    return code;
  };
  if ((e = cudaMemsetAsync(s->base + L.off_field, 0, L.field_bytes, s->stream)) != cudaSuccess ||
      (e = cudaMemsetAsync(sc, 0, 512, s->stream)) != cudaSuccess) {
    cuda_fail(s, e, "cudaMemsetAsync");
    return bail(GP_ERR_CUDA);
  }
  if ((rc = upload_tables(s)) != GP_OK) return bail(rc);
  if ((rc = set_scale_one(s)) != GP_OK) return bail(rc);
  size_t smax = 0;
  for (int m = 0; m < 2; ++m)
    for (int a = 0; a < 3; ++a) smax = std::max(smax, L.geom[m][a].smem);
  // The attribute is per kernel and process-wide: only ever raise it, so that a
  // smaller solver created later cannot lower it under a larger one.
  static size_t smem_set[2] = {0, 0};
  const int pi = L.rbytes == 8 ? 0 : 1;
  e = cudaSuccess;
  if (smax > smem_set[pi]) {
    e = pi == 0 ? gpk::sweep_set_smem_limits<double>(smax) : gpk::sweep_set_smem_limits<float>(smax);
    if (e == cudaSuccess) smem_set[pi] = smax;
  }
  if (e != cudaSuccess) {
    cuda_fail(s, e, "cudaFuncSetAttribute");
    return bail(GP_ERR_CUDA);
  }
  if ((rc = encode_maps(s)) != GP_OK) return bail(rc);
  // FP64 fields use the line-streaming sweeps unless the tile kernels are forced;
  // the z sweep's norm takes one partial per block
  if (L.rbytes == 8 && !force_tile() &&
      gpk::sweep64_blocks(2, p->nx, p->ny, p->nz) <= (long long)L.npartials) {
    if ((e = gpk::sweep64_prepare()) != cudaSuccess) {
      cuda_fail(s, e, "cudaFuncSetAttribute");
      return bail(GP_ERR_CUDA);
    }
    s->line64 = true;
  }
  fill_sweep_params(s);
  if ((e = cudaStreamSynchronize(s->stream)) != cudaSuccess) {
    cuda_fail(s, e, "cudaStreamSynchronize");
    return bail(GP_ERR_CUDA);
  }
  *out = s;
  return GP_OK;
}

cudaEvent_t take_event(gp_solver* s) {
  if (!s->pool.empty()) {
    cudaEvent_t ev = s->pool.back();
    s->pool.pop_back();
    return ev;
  }
  cudaEvent_t ev = nullptr;
  cudaEventCreate(&ev);
  return ev;
}

// NVTX range around a host-side call (shows each sweep launch and step call on a
// profiler's timeline; a no-op unless a tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

template <class R> int run_sweep(gp_solver* s, int axis) {
  static const char* const kNames[3] = {"gp sweep x", "gp sweep y", "gp sweep z"};
  NvtxRange range(kNames[axis]);
  const int m = s->is_complex ? 1 : 0;
  SweepParams q = s->sp[m][axis];
  if (axis == 0 && s->kinetic_only) q.pw = 0;
  const size_t smem = s->L.geom[m][axis].smem;
  TimedLaunch tl{nullptr, nullptr, axis};
  if (s->timing) {
    tl.start = take_event(s);
    tl.stop = take_event(s);
    GP_CUDA(s, cudaEventRecord(tl.start, s->stream));
  }
  cudaError_t e;
  if (axis == 0 && q.band_w && q.band_reg)
    e = gpk::launch_sweep_x_reg(q, m == 1, s->fast_grid[m][0], s->stream);
  else if (axis == 0 && q.band_w)
    e = gpk::launch_sweep_x_band(q, m == 1, s->fast_grid[m][0], s->stream);
  else if (q.band_w)
    e = gpk::launch_sweep_band_line(axis, q, m == 1, s->fast_grid[m][axis], s->stream);
  else if (q.trunc)
    e = gpk::launch_sweep_fast(axis, q, m == 1, s->fast_grid[m][axis], s->stream);
  else if (s->line64)
    e = gpk::launch_sweep64(axis, q, m == 1, s->stream);
  else if (axis == 0)
    e = gpk::launch_sweep_x<R>(q, m == 1, smem, s->stream);
  else if (axis == 1)
    e = gpk::launch_sweep_y<R>(s->tmap[m][1], q, m == 1, smem, s->stream);
  else
    e = gpk::launch_sweep_z<R>(s->tmap[m][2], q, m == 1, smem, s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "sweep launch");
  if (s->timing) {
    GP_CUDA(s, cudaEventRecord(tl.stop, s->stream));
    s->pending.push_back(tl);
  }
  return GP_OK;
}

// One Lie step launched directly: the three sweeps (2D: x, y, the staging copy and
// the norm pass).
template <class R> int lie_step_direct(gp_solver* s) {
  const bool two_d = s->prm.nz == 1;
  {
    for (int a = 0; a < 3; ++a) {
      if (a == 2 && two_d) {
        // 2D: no z sweep.  A fast y sweep wrote the staging area: copy it back; then
        // imaginary time renormalises with a norm pass over the plane
        const int m = s->is_complex ? 1 : 0;
        if (s->sp[m][1].trunc || s->sp[m][1].band_w)
          GP_CUDA(s, cudaMemcpyAsync(s->field, s->staging,
                                     (size_t)s->L.pitch[m] * s->L.rbytes * (m + 1) * s->prm.ny,
                                     cudaMemcpyDeviceToDevice, s->stream));
        if (!s->is_complex) {
          FieldParams f = field_params(s);
          f.out = s->scale;
          const cudaError_t e = gpk::launch_norm_to_scale<R>(f, s->stream);
          if (e != cudaSuccess) return cuda_fail(s, e, "norm");
        }
        continue;
      }
      const int rc = run_sweep<R>(s, a);
      if (rc != GP_OK) return rc;
    }
  }
  return GP_OK;
}

void drop_step_graphs(gp_solver* s) {
  for (auto* set : {s->step_exec, s->strang_exec})
    for (int m = 0; m < 2; ++m) {
      if (set[m]) cudaGraphExecDestroy(set[m]);
      set[m] = nullptr;
    }
}

// True when the solver's stream is being captured by the caller: a step then records
// its launches into the caller's graph directly.
bool caller_capturing(const gp_solver* s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s->stream, &st) != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return st != cudaStreamCaptureStatusNone;
}

// Capture the launches fn makes on s->stream into *exec, on the side stream; on any
// failure the solver falls back to direct launches for good.
template <class Fn> void capture_graph(gp_solver* s, cudaGraphExec_t* exec, Fn fn) {
  if (!s->cap_stream &&
      cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    s->cap_stream = nullptr;
    s->step_graph = false;
    return;
  }
  const cudaStream_t orig = s->stream;
  const std::string saved_err = s->err;
  s->stream = s->cap_stream;
  cudaGraph_t g = nullptr;
  bool ok = cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  const int rc = ok ? fn() : GP_OK;
  if (ok) ok = cudaStreamEndCapture(s->cap_stream, &g) == cudaSuccess && rc == GP_OK;
  s->stream = orig;
  if (ok) ok = cudaGraphInstantiate(exec, g, 0) == cudaSuccess;
  if (g) cudaGraphDestroy(g);
  if (!ok) {
    cudaGetLastError();
    *exec = nullptr;
    s->step_graph = false;
    s->err = saved_err;
  }
}

// nsteps Lie steps.  A single step (the usual call between reads of the state)
// replays the step's graph: one submission instead of separate launches starts the
// step about 2 us sooner.  Longer runs launch directly, so that each step's first
// sweep overlaps the previous step's last through programmatic dependent launch
// (graphs replayed back to back would serialise there).  The graph holds the sweep
// parameters by value: gp_set_g drops it.
template <class R> int lie_steps(gp_solver* s, long nsteps) {
  if (nsteps == 1 && s->step_graph && !s->timing && !s->kinetic_only && !caller_capturing(s)) {
    const int m = s->is_complex ? 1 : 0;
    if (!s->step_exec[m]) capture_graph(s, &s->step_exec[m], [s] { return lie_step_direct<R>(s); });
    if (s->step_exec[m]) {
      GP_CUDA(s, cudaGraphLaunch(s->step_exec[m], s->stream));
      return GP_OK;
    }
  }
  for (long t = 0; t < nsteps; ++t) {
    const int rc = lie_step_direct<R>(s);
    if (rc != GP_OK) return rc;
  }
  return GP_OK;
}

// One kinetic-only step: the three sweeps, the x sweep applying only the pending factor.
template <class R> int kinetic_step(gp_solver* s) {
  s->kinetic_only = true;
  const int rc = lie_steps<R>(s, 1);
  s->kinetic_only = false;
  return rc;
}

int set_scale_one(gp_solver* s);

// Half pointwise substep over the field (Strang): apply_scale applies the pending
// factor first (and then resets it to 1 unless norm sets it); norm makes the result's
// 1 / sqrt(norm) the pending factor.
template <class R> int half_pointwise(gp_solver* s, bool apply_scale, bool norm) {
  const int m = s->is_complex ? 1 : 0;
  FieldParams f = field_params(s);
  f.out = s->scale;
  unsigned char* coef = s->base + s->L.off_coef;
  cudaError_t e = gpk::launch_half_pointwise<R>(f, m == 1, coef + s->L.fxh_off[m],
                                                coef + s->L.fyzh_off[m], 0.5 * s->prm.dt * s->g,
                                                apply_scale, norm, s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "half pointwise");
  if (apply_scale && !norm) return set_scale_one(s);
  return GP_OK;
}

// Strang steps psi <- P(dt/2) K(dt) P(dt/2) psi (imaginary time: then renormalised).
// Real time: |psi| is invariant under the pointwise phase, so P(dt/2) P(dt/2) = P(dt)
// and n steps are P(dt/2), K, n-1 fused Lie steps, P(dt/2).  Imaginary time: each
// step is P(dt/2) (pending factor applied), K, P(dt/2) with its norm.
template <class R> int strang_steps_direct(gp_solver* s, long nsteps) {
  if (nsteps == 0) return GP_OK;
  int rc;
  if (s->is_complex) {
    if ((rc = half_pointwise<R>(s, true, false)) != GP_OK) return rc;
    if ((rc = kinetic_step<R>(s)) != GP_OK) return rc;
    if ((rc = lie_steps<R>(s, nsteps - 1)) != GP_OK) return rc;
    return half_pointwise<R>(s, true, false);
  }
  for (long t = 0; t < nsteps; ++t) {
    if ((rc = half_pointwise<R>(s, true, false)) != GP_OK) return rc;
    if ((rc = kinetic_step<R>(s)) != GP_OK) return rc;
    if ((rc = half_pointwise<R>(s, false, true)) != GP_OK) return rc;
  }
  return GP_OK;
}

// A single Strang step replays its graph, like a single Lie step.
template <class R> int strang_steps(gp_solver* s, long nsteps) {
  if (nsteps == 1 && s->step_graph && !s->timing && !caller_capturing(s)) {
    const int m = s->is_complex ? 1 : 0;
    if (!s->strang_exec[m])
      capture_graph(s, &s->strang_exec[m], [s] { return strang_steps_direct<R>(s, 1); });
    if (s->strang_exec[m]) {
      GP_CUDA(s, cudaGraphLaunch(s->strang_exec[m], s->stream));
      return GP_OK;
    }
  }
  return strang_steps_direct<R>(s, nsteps);
}

template <class R> int steps(gp_solver* s, long nsteps) {
  return s->split == GP_SPLIT_STRANG ? strang_steps<R>(s, nsteps) : lie_steps<R>(s, nsteps);
}

// Make the solver's stream wait for an overlapped read still copying its snapshot.
void wait_copies(gp_solver* s) {
  for (int h = 0; h < 2; ++h)
    if (s->copy_pending[h]) {
      cudaStreamWaitEvent(s->stream, s->copy_done[h], 0);
      s->copy_pending[h] = false;
    }
}

int set_scale_one(gp_solver* s);
int reset_steps(gp_solver* s);

// The field of a pending overlapped write (gp_set_psi_f32_async) into the solver: the
// solver stream waits for its host-to-device copy, moves it from its half of put_buf
// into the field (pitched rows, pad columns zero) and frees that half.  Every call
// that reads or writes the field runs this first.
int take_put(gp_solver* s) {
  if (!s->put_pending) return GP_OK;
  s->put_pending = false;
  GP_CUDA(s, cudaStreamWaitEvent(s->stream, s->put_ready, 0));
  s->is_complex = s->put_complex;
  FieldParams f = field_params(s);
  f.psi = s->field;
  const size_t npts = (size_t)s->prm.nx * s->prm.ny * s->prm.nz;
  const float* src = static_cast<const float*>(s->put_buf) + (size_t)s->put_half * 2 * npts;
  GP_CUDA(s, gpk::launch_import_f32(f, s->is_complex, src, s->stream));
  GP_CUDA(s, cudaEventRecord(s->put_free[s->put_half], s->stream));
  const int rc = set_scale_one(s);
  return rc != GP_OK ? rc : reset_steps(s);
}

int check_status(gp_solver* s) {
  int st = 0;
  GP_CUDA(s, cudaMemcpyAsync(&st, s->status, sizeof st, cudaMemcpyDeviceToHost, s->stream));
  GP_CUDA(s, cudaStreamSynchronize(s->stream));
  if (st == 0) return GP_OK;
  GP_CUDA(s, cudaMemsetAsync(s->status, 0, sizeof(int), s->stream));
  if (st & gpk::kStatusBounds)
    return fail(s, GP_ERR_BOUNDS, "a kernel's bounds check found an index outside its buffer");
  if (st & gpk::kStatusTimeout)
    return fail(s, GP_ERR_TIMEOUT, "a kernel's bounded wait on its tile copy ran out");
  return fail(s, GP_ERR_NONFINITE, "the norm became non-finite or zero");
}

bool is_f64(const gp_solver* s) { return s->L.rbytes == 8; }

int promote_to_complex(gp_solver* s) {
  FieldParams f = field_params(s);  // still the real layout
  cudaError_t e = is_f64(s) ? gpk::launch_export<double>(f, s->staging, false, true, s->stream)
                            : gpk::launch_export<float>(f, s->staging, false, true, s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "export");
  s->is_complex = true;
  f = field_params(s);
  e = is_f64(s) ? gpk::launch_import<double>(f, s->staging, true, s->stream)
                : gpk::launch_import<float>(f, s->staging, true, s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "import");
  return set_scale_one(s);
}

}  // namespace

// =================================================================== C ABI

extern "C" {

int gp_units_g(double natoms, double a_s_bohr, double l_osc_m, double* g) {
  constexpr double kBohr = 5.29177210903e-11;   // m, CODATA 2018
  if (!g || !(natoms >= 0.0) || !std::isfinite(natoms) || !std::isfinite(a_s_bohr) ||
      !(l_osc_m > 0.0) || !std::isfinite(l_osc_m)) {
    g_create_error = "units: natoms >= 0, a_s finite and l_osc > 0 required";
    return GP_ERR_ARG;
  }
  *g = 4.0 * kPi * natoms * (a_s_bohr * kBohr) / l_osc_m;
  return GP_OK;
}

int gp_units_l_osc(double mass_amu, double omega, double* l_osc_m) {
  constexpr double kHbar = 1.054571817e-34;     // J s (exact by the 2019 SI)
  constexpr double kAmu = 1.66053906660e-27;    // kg, CODATA 2018
  if (!l_osc_m || !(mass_amu > 0.0) || !std::isfinite(mass_amu) || !(omega > 0.0) ||
      !std::isfinite(omega)) {
    g_create_error = "units: mass and omega must be finite and > 0";
    return GP_ERR_ARG;
  }
  *l_osc_m = std::sqrt(kHbar / (mass_amu * kAmu * omega));
  return GP_OK;
}

int gp_workspace_bytes(const gp_params* p, size_t* bytes) {
  if (!bytes) {
    g_create_error = "bytes is NULL";
    return GP_ERR_ARG;
  }
  if (const char* why = check_params(p)) {
    g_create_error = why;
    return GP_ERR_ARG;
  }
  Layout L;
  if (const char* why = compute_layout(p, &L)) {
    g_create_error = why;
    return GP_ERR_ARG;
  }
  *bytes = L.total;
  return GP_OK;
}

int gp_create(const gp_params* p, void* stream, gp_solver** out) {
  return create_impl(p, nullptr, 0, stream, out);
}

int gp_create_on(const gp_params* p, void* dev_buf, size_t bytes, void* stream, gp_solver** out) {
  if (!dev_buf) {
    g_create_error = "dev_buf is NULL";
    if (out) *out = nullptr;
    return GP_ERR_ARG;
  }
  return create_impl(p, dev_buf, bytes, stream, out);
}

void gp_destroy(gp_solver* s) {
  if (!s) return;
  if (s->stream || s->base) cudaStreamSynchronize(s->stream);
  if (s->copy_stream) {
    cudaStreamSynchronize(s->copy_stream);
    cudaStreamDestroy(s->copy_stream);
  }
  if (s->copy_ready) cudaEventDestroy(s->copy_ready);
  for (auto ev : s->copy_done)
    if (ev) cudaEventDestroy(ev);
  if (s->export_buf) cudaFree(s->export_buf);
  if (s->put_stream) {
    cudaStreamSynchronize(s->put_stream);
    cudaStreamDestroy(s->put_stream);
  }
  if (s->put_ready) cudaEventDestroy(s->put_ready);
  for (auto ev : s->put_free)
    if (ev) cudaEventDestroy(ev);
  if (s->put_buf) cudaFree(s->put_buf);
  for (auto& t : s->pending) {
    cudaEventDestroy(t.start);
    cudaEventDestroy(t.stop);
  }
  for (auto ev : s->pool) cudaEventDestroy(ev);
  drop_step_graphs(s);
  if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
  if (s->owns && s->base) cudaFree(s->base);
  delete s;
}

int gp_init_gaussian(gp_solver* s, double wx, double wy, double wz) {
  if (!s) return GP_ERR_ARG;
  if (const int rc_ = take_put(s)) return rc_;   // a pending overlapped write first
  if (!(wx > 0) || !(wy > 0) || !(wz > 0) || !std::isfinite(wx) || !std::isfinite(wy) ||
      !std::isfinite(wz))
    return fail(s, GP_ERR_ARG, "Gaussian frequencies must be finite and > 0");
  s->is_complex = false;
  FieldParams f = field_params(s);
  f.out = s->scale;
  cudaError_t e = is_f64(s) ? gpk::launch_init_gaussian<double>(f, wx, wy, wz, s->stream)
                            : gpk::launch_init_gaussian<float>(f, wx, wy, wz, s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "init_gaussian");
  e = is_f64(s) ? gpk::launch_norm_to_scale<double>(f, s->stream)
                : gpk::launch_norm_to_scale<float>(f, s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "norm");
  return reset_steps(s);
}

int gp_set_psi(gp_solver* s, const double* host, int is_complex) {
  if (!s || !host || (is_complex != 0 && is_complex != 1)) return s ? fail(s, GP_ERR_ARG, "bad arguments") : GP_ERR_ARG;
  if (const int rc_ = take_put(s)) return rc_;   // a pending overlapped write first
  const size_t N = (size_t)s->prm.nx * s->prm.ny * s->prm.nz;
  GP_CUDA(s, cudaMemcpyAsync(s->staging, host, N * 8 * (is_complex ? 2 : 1),
                             cudaMemcpyHostToDevice, s->stream));
  s->is_complex = is_complex == 1;
  const FieldParams f = field_params(s);
  cudaError_t e = is_f64(s) ? gpk::launch_import<double>(f, s->staging, s->is_complex, s->stream)
                            : gpk::launch_import<float>(f, s->staging, s->is_complex, s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "import");
  const int rc = set_scale_one(s);
  return rc != GP_OK ? rc : reset_steps(s);
}

int gp_get_psi(gp_solver* s, double* host, int as_complex) {
  if (!s || !host || (as_complex != 0 && as_complex != 1)) return s ? fail(s, GP_ERR_ARG, "bad arguments") : GP_ERR_ARG;
  if (const int rc_ = take_put(s)) return rc_;   // a pending overlapped write first
  if (s->is_complex && !as_complex)
    return fail(s, GP_ERR_STATE, "the field is complex; request it with as_complex = 1");
  wait_copies(s);
  const size_t N = (size_t)s->prm.nx * s->prm.ny * s->prm.nz;
  const FieldParams f = field_params(s);
  cudaError_t e = is_f64(s)
                      ? gpk::launch_export<double>(f, s->staging, s->is_complex, as_complex == 1, s->stream)
                      : gpk::launch_export<float>(f, s->staging, s->is_complex, as_complex == 1, s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "export");
  GP_CUDA(s, cudaMemcpyAsync(host, s->staging, N * 8 * (as_complex ? 2 : 1), cudaMemcpyDeviceToHost,
                             s->stream));
  return check_status(s);
}

int gp_set_psi_f32(gp_solver* s, const float* host, int is_complex) {
  if (!s || !host || (is_complex != 0 && is_complex != 1)) return s ? fail(s, GP_ERR_ARG, "bad arguments") : GP_ERR_ARG;
  if (is_f64(s)) return fail(s, GP_ERR_ARG, "FP32 host I/O needs an FP32 solver; use gp_set_psi");
  if (const int rc_ = take_put(s)) return rc_;   // a pending overlapped write first
  s->is_complex = is_complex == 1;
  const int m = is_complex;
  const size_t eb = (size_t)4 * (m + 1), pitch = (size_t)s->L.pitch[m] * eb, row = (size_t)s->prm.nx * eb;
  const size_t rows = (size_t)s->prm.ny * s->prm.nz;
  if (pitch == row) {   // one contiguous host copy
    GP_CUDA(s, cudaMemcpyAsync(s->field, host, rows * row, cudaMemcpyHostToDevice, s->stream));
  } else {              // contiguous host copy to the staging area, pitched copy on the device
    GP_CUDA(s, cudaMemcpyAsync(s->staging, host, rows * row, cudaMemcpyHostToDevice, s->stream));
    GP_CUDA(s, cudaMemcpy2DAsync(s->field, pitch, s->staging, row, row, rows, cudaMemcpyDeviceToDevice,
                                 s->stream));
    GP_CUDA(s, cudaMemset2DAsync(static_cast<unsigned char*>(s->field) + row, pitch, 0, pitch - row, rows,
                                 s->stream));   // pad columns stay zero
  }
  const int rc = set_scale_one(s);
  return rc != GP_OK ? rc : reset_steps(s);
}

int gp_set_psi_f32_async(gp_solver* s, const float* host, int is_complex) {
  if (!s || !host || (is_complex != 0 && is_complex != 1)) return s ? fail(s, GP_ERR_ARG, "bad arguments") : GP_ERR_ARG;
  if (is_f64(s)) return fail(s, GP_ERR_ARG, "FP32 host I/O needs an FP32 solver; use gp_set_psi");
  if (!s->put_stream) {   // the put stream and its three events, all or none
    cudaStream_t ps = nullptr;
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    cudaError_t e = cudaStreamCreateWithFlags(&ps, cudaStreamNonBlocking);
    for (int q = 0; q < 3 && e == cudaSuccess; ++q) e = cudaEventCreateWithFlags(&ev[q], cudaEventDisableTiming);
    if (e != cudaSuccess) {
      for (auto x : ev)
        if (x) cudaEventDestroy(x);
      if (ps) cudaStreamDestroy(ps);
      return cuda_fail(s, e, "put stream");
    }
    s->put_stream = ps;
    s->put_ready = ev[0];
    s->put_free[0] = ev[1];
    s->put_free[1] = ev[2];
    GP_CUDA(s, cudaEventRecord(s->put_free[0], s->stream));
    GP_CUDA(s, cudaEventRecord(s->put_free[1], s->stream));
  }
  const size_t npts = (size_t)s->prm.nx * s->prm.ny * s->prm.nz;
  if (!s->put_buf && cudaMalloc(&s->put_buf, 16 * npts) != cudaSuccess) {   // two packed complex fields
    cudaGetLastError();
    s->put_buf = nullptr;
    return fail(s, GP_ERR_NOMEM, "no device memory for the buffers of overlapped writes");
  }
  // a write still waiting to be taken is superseded: take it first
  int rc = take_put(s);
  if (rc != GP_OK) return rc;
  const int h = s->put_next;
  s->put_next ^= 1;
  GP_CUDA(s, cudaStreamWaitEvent(s->put_stream, s->put_free[h], 0));   // its half was moved
  float* dst = static_cast<float*>(s->put_buf) + (size_t)h * 2 * npts;
  GP_CUDA(s, cudaMemcpyAsync(dst, host, (size_t)4 * (is_complex + 1) * npts, cudaMemcpyHostToDevice,
                             s->put_stream));
  GP_CUDA(s, cudaEventRecord(s->put_ready, s->put_stream));
  s->put_pending = true;
  s->put_complex = is_complex == 1;
  s->put_half = h;
  return GP_OK;
}

int gp_get_psi_f32(gp_solver* s, float* host, int as_complex) {
  if (!s || !host || (as_complex != 0 && as_complex != 1)) return s ? fail(s, GP_ERR_ARG, "bad arguments") : GP_ERR_ARG;
  if (is_f64(s)) return fail(s, GP_ERR_ARG, "FP32 host I/O needs an FP32 solver; use gp_get_psi");
  if (const int rc_ = take_put(s)) return rc_;   // a pending overlapped write first
  if (as_complex != (s->is_complex ? 1 : 0))
    return fail(s, GP_ERR_STATE, "as_complex must match the field (0: real, 1: complex)");
  wait_copies(s);
  const int m = as_complex;
  // the field times the pending factor, packed into the staging area (the field and
  // its factor stay as they are: a read does not change the next steps' bits)
  const size_t bytes = (size_t)4 * (m + 1) * s->prm.nx * s->prm.ny * s->prm.nz;
  float* packed = reinterpret_cast<float*>(s->staging);
  const cudaError_t e = gpk::launch_export_f32(field_params(s), m == 1, packed, s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "export");
  GP_CUDA(s, cudaMemcpyAsync(host, packed, bytes, cudaMemcpyDeviceToHost, s->stream));
  return check_status(s);
}

int gp_get_psi_f32_async(gp_solver* s, float* host, int as_complex) {
  if (!s || !host || (as_complex != 0 && as_complex != 1)) return s ? fail(s, GP_ERR_ARG, "bad arguments") : GP_ERR_ARG;
  if (is_f64(s)) return fail(s, GP_ERR_ARG, "FP32 host I/O needs an FP32 solver; use gp_get_psi");
  if (const int rc_ = take_put(s)) return rc_;   // a pending overlapped write first
  if (as_complex != (s->is_complex ? 1 : 0))
    return fail(s, GP_ERR_STATE, "as_complex must match the field (0: real, 1: complex)");
  if (!s->copy_stream) {   // the copy stream and its three events, all or none
    cudaStream_t cs = nullptr;
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    for (int q = 0; q < 3 && e == cudaSuccess; ++q) e = cudaEventCreateWithFlags(&ev[q], cudaEventDisableTiming);
    if (e != cudaSuccess) {
      for (auto x : ev)
        if (x) cudaEventDestroy(x);
      if (cs) cudaStreamDestroy(cs);
      return cuda_fail(s, e, "copy stream");
    }
    s->copy_stream = cs;
    s->copy_ready = ev[0];
    s->copy_done[0] = ev[1];
    s->copy_done[1] = ev[2];
  }
  const size_t npts = (size_t)s->prm.nx * s->prm.ny * s->prm.nz;
  if (!s->export_buf && cudaMalloc(&s->export_buf, 16 * npts) != cudaSuccess) {   // two packed complex fields
    cudaGetLastError();
    s->export_buf = nullptr;
    return fail(s, GP_ERR_NOMEM, "no device memory for the snapshots of overlapped reads");
  }
  // this read's half of the snapshot buffer; its previous read may still be copying
  const int h = s->export_next;
  s->export_next ^= 1;
  if (s->copy_pending[h]) {
    GP_CUDA(s, cudaStreamWaitEvent(s->stream, s->copy_done[h], 0));
    s->copy_pending[h] = false;
  }
  const int m = as_complex;
  const size_t bytes = (size_t)4 * (m + 1) * npts;
  float* snap = static_cast<float*>(s->export_buf) + (size_t)h * 2 * npts;
  const cudaError_t e = gpk::launch_export_f32(field_params(s), m == 1, snap, s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "export");
  GP_CUDA(s, cudaEventRecord(s->copy_ready, s->stream));
  GP_CUDA(s, cudaStreamWaitEvent(s->copy_stream, s->copy_ready, 0));
  GP_CUDA(s, cudaMemcpyAsync(host, snap, bytes, cudaMemcpyDeviceToHost, s->copy_stream));
  GP_CUDA(s, cudaEventRecord(s->copy_done[h], s->copy_stream));
  s->copy_pending[h] = true;
  return GP_OK;
}

int gp_step_imag(gp_solver* s, long nsteps) {
  if (!s || nsteps < 0) return s ? fail(s, GP_ERR_ARG, "nsteps must be >= 0") : GP_ERR_ARG;
  if (const int rc_ = take_put(s)) return rc_;   // a pending overlapped write first
  if (s->is_complex) return fail(s, GP_ERR_STATE, "imaginary-time steps need a real field");
  NvtxRange range("gp_step_imag");
  return is_f64(s) ? steps<double>(s, nsteps) : steps<float>(s, nsteps);
}

int gp_step_real(gp_solver* s, long nsteps) {
  if (!s || nsteps < 0) return s ? fail(s, GP_ERR_ARG, "nsteps must be >= 0") : GP_ERR_ARG;
  if (const int rc_ = take_put(s)) return rc_;   // a pending overlapped write first
  if (!s->is_complex) {
    const int rc = promote_to_complex(s);
    if (rc != GP_OK) return rc;
  }
  NvtxRange range("gp_step_real");
  return is_f64(s) ? steps<double>(s, nsteps) : steps<float>(s, nsteps);
}

int gp_set_splitting(gp_solver* s, int scheme) {
  if (!s) return GP_ERR_ARG;
  if (scheme != GP_SPLIT_LIE && scheme != GP_SPLIT_STRANG)
    return fail(s, GP_ERR_ARG, "scheme must be GP_SPLIT_LIE or GP_SPLIT_STRANG");
  s->split = scheme;
  return GP_OK;
}

int gp_set_g(gp_solver* s, double g) {
  if (!s) return GP_ERR_ARG;
  if (!std::isfinite(g)) return fail(s, GP_ERR_ARG, "g must be finite");
  s->g = g;
  for (int m = 0; m < 2; ++m)
    for (int a = 0; a < 3; ++a) {
      s->sp[m][a].g = g;
      s->sp[m][a].band_dtg = (float)(s->sp[m][a].dt * g);
    }
  drop_step_graphs(s);   // they hold the old parameters
  return GP_OK;
}

int gp_set_wait_limit(gp_solver* s, long long first_wait_ns) {
  if (!s) return GP_ERR_ARG;
  const unsigned long long ns =
      first_wait_ns < 0 ? gpk::kWaitLimitNs
                        : std::min<unsigned long long>((unsigned long long)first_wait_ns,
                                                       gpk::kWaitLimitNs);
  for (int m = 0; m < 2; ++m)
    for (int a = 0; a < 3; ++a) s->sp[m][a].wait_ns = ns;
  drop_step_graphs(s);   // they hold the old parameters
  return GP_OK;
}

int gp_get_g(const gp_solver* s, double* g) {
  if (!s || !g) return GP_ERR_ARG;
  *g = s->g;
  return GP_OK;
}

int gp_observables(gp_solver* s, gp_obs* out) {
  if (!s || !out) return s ? fail(s, GP_ERR_ARG, "out is NULL") : GP_ERR_ARG;
  if (const int rc_ = take_put(s)) return rc_;   // a pending overlapped write first
  wait_copies(s);
  const FieldParams f = field_params(s);
  cudaError_t e = is_f64(s) ? gpk::launch_observables<double>(f, s->is_complex, s->stream)
                            : gpk::launch_observables<float>(f, s->is_complex, s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "observables");
  double o[10];
  GP_CUDA(s, cudaMemcpyAsync(o, s->obs, sizeof o, cudaMemcpyDeviceToHost, s->stream));
  const int rc = check_status(s);
  if (rc != GP_OK) return rc;
  out->norm = o[0];
  out->mu = o[1];
  out->energy = o[2];
  out->ekin = o[3];
  out->epot = o[4];
  out->eint = o[5];
  out->rms_x = o[6];
  out->rms_y = o[7];
  out->rms_z = o[8];
  out->rms_r = o[9];
  return GP_OK;
}

int gp_density2d(gp_solver* s, int plane, double* out) {
  if (!s || !out || plane < 0 || plane > 2) return s ? fail(s, GP_ERR_ARG, "bad arguments") : GP_ERR_ARG;
  if (const int rc_ = take_put(s)) return rc_;   // a pending overlapped write first
  wait_copies(s);
  const gp_params& p = s->prm;
  const FieldParams f = field_params(s);
  cudaError_t e = is_f64(s) ? gpk::launch_density2d<double>(f, s->is_complex, plane, s->staging, s->stream)
                            : gpk::launch_density2d<float>(f, s->is_complex, plane, s->staging, s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "density2d");
  const size_t n = plane == 0 ? (size_t)p.nx * p.ny : plane == 1 ? (size_t)p.nx * p.nz
                                                                 : (size_t)p.ny * p.nz;
  GP_CUDA(s, cudaMemcpyAsync(out, s->staging, n * 8, cudaMemcpyDeviceToHost, s->stream));
  return check_status(s);
}

int gp_density1d(gp_solver* s, int axis, double* out) {
  if (!s || !out || axis < 0 || axis > 2) return s ? fail(s, GP_ERR_ARG, "bad arguments") : GP_ERR_ARG;
  if (const int rc_ = take_put(s)) return rc_;   // a pending overlapped write first
  wait_copies(s);
  const gp_params& p = s->prm;
  const FieldParams f = field_params(s);
  const int plane = axis == 2 ? 1 : 0;  // x, y from the xy plane; z from the xz plane
  cudaError_t e = is_f64(s) ? gpk::launch_density2d<double>(f, s->is_complex, plane, s->staging, s->stream)
                            : gpk::launch_density2d<float>(f, s->is_complex, plane, s->staging, s->stream);
  if (e != cudaSuccess) return cuda_fail(s, e, "density2d");
  double* red = s->staging + (size_t)p.nx * std::max(p.ny, p.nz);
  if (axis == 0)
    e = gpk::launch_cols_sum(s->staging, p.ny, p.nx, p.dy, red, s->stream);   // sum over y
  else if (axis == 1)
    e = gpk::launch_rows_sum(s->staging, p.ny, p.nx, p.dx, red, s->stream);   // sum over x
  else
    e = gpk::launch_rows_sum(s->staging, p.nz, p.nx, p.dx, red, s->stream);   // sum over x
  if (e != cudaSuccess) return cuda_fail(s, e, "density1d");
  const size_t n = axis == 0 ? p.nx : axis == 1 ? p.ny : p.nz;
  GP_CUDA(s, cudaMemcpyAsync(out, red, n * 8, cudaMemcpyDeviceToHost, s->stream));
  return check_status(s);
}

int gp_sync(gp_solver* s) {
  if (!s) return GP_ERR_ARG;
  if (const int rc_ = take_put(s)) return rc_;   // a pending overlapped write first
  wait_copies(s);
  resolve_scale(s);   // a deferred norm's non-finite flag is set where it is summed
  return check_status(s);
}

int gp_set_timing(gp_solver* s, int enable) {
  if (!s) return GP_ERR_ARG;
  s->timing = enable != 0;
  return GP_OK;
}

int gp_get_timing(gp_solver* s, double ms[3], long long launches[3]) {
  if (!s || !ms || !launches) return GP_ERR_ARG;
  GP_CUDA(s, cudaStreamSynchronize(s->stream));
  for (int a = 0; a < 3; ++a) {
    ms[a] = 0.0;
    launches[a] = 0;
  }
  for (auto& t : s->pending) {
    float el = 0.f;
    GP_CUDA(s, cudaEventElapsedTime(&el, t.start, t.stop));
    ms[t.axis] += el;
    launches[t.axis] += 1;
    s->pool.push_back(t.start);
    s->pool.push_back(t.stop);
  }
  s->pending.clear();
  return GP_OK;
}

int gp_get_info(const gp_solver* s, long long info[8]) {
  if (!s || !info) return GP_ERR_ARG;
  const int m = s->is_complex ? 1 : 0;
  info[0] = s->L.pitch[m];
  info[1] = m;
  info[2] = s->L.geom[m][0].lines;
  info[3] = s->L.geom[m][1].lines;
  info[4] = s->L.geom[m][2].lines;
  info[5] = (long long)s->L.total;
  info[6] = 0;
  int wmax = 0;
  for (int a = 0; a < 3; ++a) {
    if (s->trunc[m][a] || s->band_w[m][a]) info[6] |= 1 << a;
    if (s->band_w[m][a]) info[6] |= 8 << a;
    wmax = std::max(wmax, s->band_w[m][a]);
  }
  info[6] |= (long long)wmax << 8;
  if (s->line64) info[6] |= 7LL << 12;
  if (s->sp[m][0].band_reg) info[6] |= 1LL << 15;
  info[7] = std::max(s->trunc[m][0], std::max(s->trunc[m][1], s->trunc[m][2]));
  return GP_OK;
}

const char* gp_last_error(const gp_solver* s) {
  return s ? s->err.c_str() : g_create_error.c_str();
}

const char* gp_strerror(int code) {
  switch (code) {
    case GP_OK: return "ok";
    case GP_ERR_ARG: return "invalid argument";
    case GP_ERR_NOMEM: return "out of device memory or buffer too small";
    case GP_ERR_CUDA: return "CUDA error";
    case GP_ERR_NONFINITE: return "non-finite or zero norm";
    case GP_ERR_TIMEOUT: return "kernel wait timed out";
    case GP_ERR_STATE: return "invalid in the current mode";
    case GP_ERR_BOUNDS: return "bounds check failed (GP_CHECK build)";
    default: return "unknown error";
  }
}

}  // extern "C"

// gp_batch.cu -- pools of resident FP32 solves stepped together (batched uneven
// solves and the serving loop): a device arena with a first-fit allocator, per-slot
// tables and descriptors, packed work lists (rows of every x line; blocks of every
// y / z line segment), one batched launch per sweep direction and mode, the step
// captured as a CUDA graph, per-slot observables and field I/O, and an autotuner over
// the launch shapes.  Every slot runs the same SSCN step as a single FP32 solver
// (paper, program summary: "Solution method") with the banded line operators of
// gp_sweeps.cu; a slot's arithmetic does not depend on which other slots are live.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/gp.h"
#include "gp_arena.h"
#include "gp_internal.h"

using gpk::BatchArgs;
using gpk::FieldParams;
using gpk::LineBlock;
using gpk::SlotDesc;
using gpk::XItem;

namespace {

constexpr size_t kAlign = 256;
constexpr int kMaxPoolSlots = 4096;
constexpr size_t kMaxSmem = 227 * 1024;   // opt-in shared memory per block
constexpr size_t kXWarpBudget = 6 * 1024;  // x: row slots of one warp for groups of rows
constexpr int kWeights = 2 * gpk::kBandHalfMax + 1;

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

using gp_arena::Arena;

// Byte layout of one slot inside the arena (offsets from the slot's start).
struct SlotGeom {
  int pitch[2] = {0, 0};       // row pitch in elements: real field, complex field
  size_t field_bytes = 0;      // sized for the complex field
  size_t off_field = 0, off_staging = 0, off_fx[2] = {}, off_fyz[2] = {}, off_otab = 0;
  size_t off_scal = 0, off_partials = 0, total = 0;
  int max_blocks_z = 0;        // z blocks of the slot at the shortest segment
};

void slot_geometry(const gp_params& p, SlotGeom* G) {
  const size_t rows = (size_t)p.ny * p.nz;
  G->pitch[0] = (int)align_up((size_t)p.nx, 4);
  G->pitch[1] = (int)align_up((size_t)p.nx, 2);
  G->field_bytes = std::max((size_t)G->pitch[0] * 4, (size_t)G->pitch[1] * 8) * rows;
  // z blocks at the shortest segment (one turn of the smallest ring, 7 points)
  int mb = 0;
  for (int m = 0; m < 2; ++m) {
    const long long cols = (long long)((p.nx + (m ? 1 : 3)) / (m ? 2 : 4)) * p.ny;
    const long long nseg = (p.nz + 6) / 7;
    mb = std::max<int>(mb, (int)((cols * nseg + 127) / 128));
  }
  G->max_blocks_z = mb;
  size_t off = 0;
  G->off_field = off;
  off = align_up(off + G->field_bytes, kAlign);
  G->off_staging = off;
  off = align_up(off + G->field_bytes, kAlign);
  for (int m = 0; m < 2; ++m) {
    G->off_fx[m] = off;
    off = align_up(off + (size_t)G->pitch[m] * 4 * (m + 1), kAlign);
    G->off_fyz[m] = off;
    off = align_up(off + rows * 4 * (m + 1), kAlign);
  }
  G->off_otab = off;
  off = align_up(off + (size_t)2 * (p.nx + p.ny + p.nz) * 8, kAlign);
  G->off_scal = off;   // scale (8), counter (4)
  off = align_up(off + 64, kAlign);
  G->off_partials = off;
  off = align_up(off + (size_t)mb * 8, kAlign);
  G->total = off;
}

struct Slot {
  bool live = false;
  gp_params prm{};
  double g = 0.0;
  int mode = 0;               // 0 imaginary time (real field), 1 real time (complex field)
  size_t off = 0;
  SlotGeom G;
  int band_w[2][3] = {};
  float wt[2][3][2 * kWeights] = {};   // kBandHalfMax-centred weights per mode and axis
};

__global__ void k_pool_set_double(double* p, double v) { *p = v; }

// real field (pitch p0) times the pending factor -> complex field (pitch p1), FP64
// product rounded once, as the single solver's hand-off through FP64 does
__global__ void k_real_to_complex(const float* __restrict__ src, int p0, float2* __restrict__ dst,
                                  int p1, int nx, long long rows, const double* scale) {
  const double s = *scale;
  for (long long r = blockIdx.x; r < rows; r += gridDim.x)
    for (int i = threadIdx.x; i < p1; i += blockDim.x)
      dst[(size_t)r * p1 + i] =
          i < nx ? make_float2((float)((double)src[(size_t)r * p0 + i] * s), 0.f) : make_float2(0.f, 0.f);
}

}  // namespace

struct gp_pool {
  int device = 0, nsm = 0;
  cudaStream_t stream = nullptr;
  bool owns_stream = false;
  unsigned char* arena = nullptr;
  size_t capacity = 0;
  Arena alloc;
  std::vector<Slot> slots;
  SlotDesc* d_desc = nullptr;
  std::vector<SlotDesc> h_desc;
  // packed work lists per mode and axis
  void* d_items[2][3] = {};
  size_t items_cap[2][3] = {};
  int nitems[2][3] = {};
  int wl[2][3] = {};           // launch half-width per mode and axis
  int slot_elems[2] = {};      // x: shared-memory row slot per mode
  size_t x_smem[2] = {};
  int x_stages_used[2] = {2, 2};
  bool x_reg[2] = {false, false};    // x sweep with rows in registers for the mode's slots
  int x_group_max[2] = {1, 1};
  int live_mode[2] = {};       // live slots per mode
  // launch shape (autotuned)
  int x_stages = 3, seg_turns = 3;
  // reductions and I/O scratch
  unsigned char* d_scratch = nullptr;   // partials | counter | obs | status
  double* d_partials = nullptr;
  unsigned int* d_counter = nullptr;
  double* d_obs = nullptr;
  int* d_status = nullptr;
  double* d_io = nullptr;
  size_t io_bytes = 0;
  // step graph
  bool use_graph = true;
  cudaGraphExec_t exec = nullptr;
  bool dirty = true;
  int launches_per_step = 0;
  std::string err = "no error";
};

namespace {

int pfail(gp_pool* P, int code, const std::string& msg) {
  if (P) P->err = msg;
  return code;
}
int pcuda(gp_pool* P, cudaError_t e, const char* where) {
  return pfail(P, GP_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}
#define PCUDA(P, call)                                  \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return pcuda((P), e_, #call); \
  } while (0)

// GP_X_REG=0 keeps the pools' x sweeps on the copy-fed kernel (A/B measurements).
bool batch_x_reg_enabled() {
  const char* v = std::getenv("GP_X_REG");
  return !(v && std::strcmp(v, "0") == 0);
}

bool slot_ok(const gp_pool* P, int slot) {
  return P && slot >= 0 && slot < (int)P->slots.size() && P->slots[slot].live;
}

unsigned char* slot_base(const gp_pool* P, const Slot& S) { return P->arena + S.off; }

FieldParams slot_field(gp_pool* P, int slot) {
  Slot& S = P->slots[slot];
  unsigned char* b = slot_base(P, S);
  FieldParams f;
  f.psi = b + S.G.off_field;
  f.nx = S.prm.nx;
  f.ny = S.prm.ny;
  f.nz = S.prm.nz;
  f.pitch = S.G.pitch[S.mode];
  f.scale = reinterpret_cast<double*>(b + S.G.off_scal);
  f.partials = P->d_partials;
  f.counter = P->d_counter;
  f.out = P->d_obs;
  f.status = P->d_status;
  f.tab = reinterpret_cast<const double*>(b + S.G.off_otab);
  f.hx = S.prm.dx;
  f.hy = S.prm.dy;
  f.hz = S.prm.dz;
  f.g = S.g;
  return f;
}

double nonlinearity_of(const gp_params& p) {
  constexpr double kPi = 3.14159265358979323846264338327950288;
  return p.use_physical ? 4.0 * kPi * p.natoms * p.a_s / p.l_osc : p.g;
}

// Tables of one slot: trap factors (FP32, separable) and FP64 V, x^2 for the
// observables; banded weights per mode and axis.  False when an axis has no band.
bool slot_tables(const gp_params& p, const SlotGeom& G, Slot* S, std::vector<unsigned char>* buf) {
  const int n[3] = {p.nx, p.ny, p.nz};
  const double h[3] = {p.dx, p.dy, p.dz};
  const double w[3] = {p.gamma, p.nu, p.lambda};
  for (int m = 0; m < 2; ++m)
    for (int a = 0; a < 3; ++a) {
      const double beta = p.dt / (4.0 * h[a] * h[a]);
      std::vector<std::complex<double>> wts;
      const int W = gpk::cn_free_row(m == 0 ? std::complex<double>(beta, 0.0)
                                            : std::complex<double>(0.0, beta), &wts);
      if (!W || n[a] < 8) return false;
      wts[W] -= 1.0;   // the kernels add the identity part separately
      S->band_w[m][a] = W;
      std::fill(std::begin(S->wt[m][a]), std::end(S->wt[m][a]), 0.f);
      for (int k = 0; k <= 2 * W; ++k) {
        const int c = gpk::kBandHalfMax - W + k;
        if (m == 0) {
          S->wt[m][a][c] = (float)wts[k].real();
        } else {
          S->wt[m][a][2 * c] = (float)wts[k].real();
          S->wt[m][a][2 * c + 1] = (float)wts[k].imag();
        }
      }
    }
  buf->assign(G.total - G.off_fx[0], 0);
  auto put = [&](size_t off, const void* v, size_t bytes) {
    std::memcpy(buf->data() + (off - G.off_fx[0]), v, bytes);
  };
  auto pot = [&](int a, int i) {
    const double x = (i - 0.5 * (n[a] - 1)) * h[a];
    return 0.5 * w[a] * w[a] * x * x;
  };
  for (int i = 0; i < p.nx; ++i) {
    const double th = p.dt * pot(0, i);
    const float e = (float)std::exp(-th), cs[2] = {(float)std::cos(th), (float)-std::sin(th)};
    put(G.off_fx[0] + (size_t)i * 4, &e, 4);
    put(G.off_fx[1] + (size_t)i * 8, cs, 8);
  }
  for (int k = 0; k < p.nz; ++k)
    for (int j = 0; j < p.ny; ++j) {
      const double th = p.dt * (pot(1, j) + pot(2, k));
      const size_t r = (size_t)k * p.ny + j;
      const float e = (float)std::exp(-th), cs[2] = {(float)std::cos(th), (float)-std::sin(th)};
      put(G.off_fyz[0] + r * 4, &e, 4);
      put(G.off_fyz[1] + r * 8, cs, 8);
    }
  const int ntot = p.nx + p.ny + p.nz;
  size_t iv = 0;
  for (int a = 0; a < 3; ++a)
    for (int i = 0; i < n[a]; ++i, ++iv) {
      const double x = (i - 0.5 * (n[a] - 1)) * h[a];
      const double V = pot(a, i), x2 = x * x;
      put(G.off_otab + iv * 8, &V, 8);
      put(G.off_otab + (ntot + iv) * 8, &x2, 8);
    }
  return true;
}

template <class T> int grow(gp_pool* P, void** d, size_t* cap, size_t count) {
  const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
  if (*cap >= bytes) return GP_OK;
  if (*d) cudaFree(*d);
  *d = nullptr;
  *cap = 0;
  PCUDA(P, cudaMalloc(d, bytes));
  *cap = bytes;
  return GP_OK;
}

void drop_graph(gp_pool* P) {
  if (P->exec) cudaGraphExecDestroy(P->exec);
  P->exec = nullptr;
}

// Descriptors, launch half-widths and work lists of the live slots.
int rebuild(gp_pool* P) {
  drop_graph(P);
  const int ns = (int)P->slots.size();
  for (int m = 0; m < 2; ++m) {
    P->live_mode[m] = 0;
    P->slot_elems[m] = 0;
    for (int a = 0; a < 3; ++a) P->wl[m][a] = 0;
  }
  for (int i = 0; i < ns; ++i) {
    const Slot& S = P->slots[i];
    if (!S.live) continue;
    const int m = S.mode;
    ++P->live_mode[m];
    P->slot_elems[m] = std::max(P->slot_elems[m], S.G.pitch[m] + 16);
    for (int a = 0; a < 3; ++a) P->wl[m][a] = std::max(P->wl[m][a], S.band_w[m][a]);
  }
  // descriptors
  for (int i = 0; i < ns; ++i) {
    const Slot& S = P->slots[i];
    SlotDesc& d = P->h_desc[i];
    std::memset(&d, 0, sizeof d);
    if (!S.live) continue;
    const int m = S.mode;
    unsigned char* b = slot_base(P, S);
    d.field = b + S.G.off_field;
    d.staging = b + S.G.off_staging;
    d.fx = b + S.G.off_fx[m];
    d.fyz = b + S.G.off_fyz[m];
    d.scale = reinterpret_cast<double*>(b + S.G.off_scal);
    d.counter = reinterpret_cast<unsigned int*>(b + S.G.off_scal + 8);
    d.partials = reinterpret_cast<double*>(b + S.G.off_partials);
    d.nx = S.prm.nx;
    d.ny = S.prm.ny;
    d.nz = S.prm.nz;
    d.pitch = S.G.pitch[m];
    for (int a = 1; a < 3; ++a) d.seg[a] = P->seg_turns * (2 * P->wl[m][a] + 1);
    d.dtg = (float)(S.prm.dt * S.g);
    d.dV = S.prm.dx * S.prm.dy * S.prm.dz;
    std::memcpy(d.wt, S.wt[m], sizeof d.wt);
  }
  PCUDA(P, cudaMemcpyAsync(P->d_desc, P->h_desc.data(), sizeof(SlotDesc) * ns,
                           cudaMemcpyHostToDevice, P->stream));
  P->launches_per_step = 0;
  for (int m = 0; m < 2; ++m) {
    const bool cplx = m == 1;
    if (!P->live_mode[m]) {
      for (int a = 0; a < 3; ++a) P->nitems[m][a] = 0;
      continue;
    }
    // x: stages that fit shared memory, rows per group per slot, rows per warp such
    // that every warp is resident at once
    // slots whose rows are EPL m <= 32 EPL points (EPL = 16 real, 8 complex elements)
    // at a half-width of 3 or 5: rows in registers, floor(32 / (nx / EPL)) rows of a
    // slot per warp pass
    const int epl = cplx ? 8 : 16;
    bool reg = batch_x_reg_enabled();
    for (int i = 0; i < ns && reg; ++i)
      if (P->slots[i].live && P->slots[i].mode == m)
        reg = gpk::batch_x_reg_fits(P->slots[i].prm.nx, P->wl[m][0], cplx);
    int rbps = 0;
    if (reg && (gpk::batch_x_reg_prepare(P->wl[m][0], cplx, &rbps) != cudaSuccess || rbps <= 0)) {
      cudaGetLastError();
      reg = false;
    }
    P->x_reg[m] = reg;
    int st = P->x_stages;
    while (st > 2 && gpk::batch_x_smem(st, 1, P->slot_elems[m], cplx) > kMaxSmem) --st;
    P->x_stages_used[m] = st;
    const size_t slot_bytes = (size_t)P->slot_elems[m] * (cplx ? 8 : 4);
    int gmax = 1;
    std::vector<int> grp(ns, 1);
    for (int i = 0; i < ns; ++i)
      if (P->slots[i].live && P->slots[i].mode == m) {
        grp[i] = gpk::x_band_group(P->slots[i].prm.nx, cplx ? 2 : 4, st, slot_bytes, kXWarpBudget);
        gmax = std::max(gmax, grp[i]);
      }
    while (gmax > 1 && gpk::batch_x_smem(st, gmax, P->slot_elems[m], cplx) > kMaxSmem) {
      --gmax;
      for (int& g : grp) g = std::min(g, gmax);
    }
    P->x_group_max[m] = gmax;
    P->x_smem[m] = gpk::batch_x_smem(st, gmax, P->slot_elems[m], cplx);
    int bps = 0;
    cudaError_t e = gpk::batch_prepare(P->wl[m][0], cplx, P->x_smem[m], &bps);
    if (e != cudaSuccess) return pcuda(P, e, "batch_prepare");
    if (bps <= 0) return pfail(P, GP_ERR_ARG, "the x rows of the widest slot do not fit shared memory");
    long long rows_tot = 0;
    for (int i = 0; i < ns; ++i)
      if (P->slots[i].live && P->slots[i].mode == m)
        rows_tot += (long long)P->slots[i].prm.ny * P->slots[i].prm.nz;
    const long long cap = reg ? (long long)P->nsm * rbps * gpk::kXRegWarps
                              : (long long)P->nsm * bps * gpk::kBatchXWarps;
    const int rpw = (int)std::max<long long>(1, (rows_tot + cap - 1) / cap);
    std::vector<XItem> xi;
    std::vector<LineBlock> lb[3];
    for (int i = 0; i < ns; ++i) {
      const Slot& S = P->slots[i];
      if (!S.live || S.mode != m) continue;
      const long long rows = (long long)S.prm.ny * S.prm.nz;
      // register rows: items of a whole number of passes of rp rows each
      const int rp = reg ? std::max(1, 32 / (S.prm.nx / epl)) : 1;
      const int ipw = reg ? (rpw + rp - 1) / rp * rp : rpw;
      for (long long r = 0; r < rows; r += ipw) {
        XItem it;
        it.slot = i;
        it.row0 = r;
        it.nrow = (int)std::min<long long>(ipw, rows - r);
        it.group = reg ? rp : grp[i];
        it.pad = 0;
        xi.push_back(it);
      }
      const int ept = cplx ? 2 : 4;
      for (int a = 1; a < 3; ++a) {
        const int n = a == 1 ? S.prm.ny : S.prm.nz;
        const long long cols = (long long)((S.prm.nx + ept - 1) / ept) * (a == 1 ? S.prm.nz : S.prm.ny);
        const int seg = P->seg_turns * (2 * P->wl[m][a] + 1);
        const long long nb = (cols * ((n + seg - 1) / seg) + 127) / 128;
        if (a == 2 && nb > S.G.max_blocks_z) return pfail(P, GP_ERR_ARG, "z blocks exceed the slot's partials");
        for (long long q = 0; q < nb; ++q) {
          LineBlock l;
          l.slot = i;
          l.blk = (int)q;
          l.nblk = (int)nb;
          l.pad = 0;
          lb[a].push_back(l);
        }
      }
    }
    int rc = grow<XItem>(P, &P->d_items[m][0], &P->items_cap[m][0], xi.size());
    if (rc != GP_OK) return rc;
    PCUDA(P, cudaMemcpyAsync(P->d_items[m][0], xi.data(), xi.size() * sizeof(XItem),
                             cudaMemcpyHostToDevice, P->stream));
    P->nitems[m][0] = (int)xi.size();
    for (int a = 1; a < 3; ++a) {
      rc = grow<LineBlock>(P, &P->d_items[m][a], &P->items_cap[m][a], lb[a].size());
      if (rc != GP_OK) return rc;
      PCUDA(P, cudaMemcpyAsync(P->d_items[m][a], lb[a].data(), lb[a].size() * sizeof(LineBlock),
                               cudaMemcpyHostToDevice, P->stream));
      P->nitems[m][a] = (int)lb[a].size();
    }
    P->launches_per_step += 3;
  }
  P->dirty = false;
  return GP_OK;
}

int launch_step(gp_pool* P) {
  for (int m = 0; m < 2; ++m) {
    if (!P->live_mode[m]) continue;
    for (int a = 0; a < 3; ++a) {
      BatchArgs b;
      b.slots = P->d_desc;
      b.items = P->d_items[m][a];
      b.nitems = P->nitems[m][a];
      b.stages = P->x_stages_used[m];
      b.group_max = P->x_group_max[m];
      b.slot_elems = P->slot_elems[m];
      b.status = P->d_status;
      b.wait_ns = gpk::kWaitLimitNs;
      b.x_reg = P->x_reg[m] ? 1 : 0;
      const int xw = b.x_reg ? gpk::kXRegWarps : gpk::kBatchXWarps;
      const int grid = a == 0 ? (b.nitems + xw - 1) / xw : b.nitems;
      const cudaError_t e = gpk::launch_batch_sweep(a, P->wl[m][a], b, m == 1, grid,
                                                    a == 0 && !b.x_reg ? P->x_smem[m] : 0, P->stream);
      if (e != cudaSuccess) return pcuda(P, e, "batched sweep launch");
    }
  }
  return GP_OK;
}

int check_status(gp_pool* P) {
  int st = 0;
  PCUDA(P, cudaMemcpyAsync(&st, P->d_status, sizeof st, cudaMemcpyDeviceToHost, P->stream));
  PCUDA(P, cudaStreamSynchronize(P->stream));
  if (st == 0) return GP_OK;
  PCUDA(P, cudaMemsetAsync(P->d_status, 0, sizeof(int), P->stream));
  if (st & gpk::kStatusTimeout) return pfail(P, GP_ERR_TIMEOUT, "a kernel's bounded wait ran out");
  return pfail(P, GP_ERR_NONFINITE, "the norm of a slot became non-finite or zero");
}

// nsteps steps of every live slot (graph replay when enabled), no status read.
int run_steps(gp_pool* P, long nsteps) {
  if (P->dirty) {
    const int rc = rebuild(P);
    if (rc != GP_OK) return rc;
  }
  if (P->launches_per_step == 0 || nsteps == 0) return GP_OK;
  if (P->use_graph && !P->exec) {
    cudaGraph_t g = nullptr;
    bool ok = cudaStreamBeginCapture(P->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    int rc = GP_OK;
    if (ok) {
      rc = launch_step(P);
      ok = cudaStreamEndCapture(P->stream, &g) == cudaSuccess && rc == GP_OK;
    }
    if (ok) ok = cudaGraphInstantiate(&P->exec, g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    if (!ok) {   // graphs unavailable here: direct launches from now on
      cudaGetLastError();
      P->exec = nullptr;
      P->use_graph = false;
    }
  }
  for (long t = 0; t < nsteps; ++t) {
    if (P->exec) {
      PCUDA(P, cudaGraphLaunch(P->exec, P->stream));
    } else {
      const int rc = launch_step(P);
      if (rc != GP_OK) return rc;
    }
  }
  return GP_OK;
}

int ensure_io(gp_pool* P, size_t bytes) {
  if (P->io_bytes >= bytes) return GP_OK;
  if (P->d_io) {
    PCUDA(P, cudaStreamSynchronize(P->stream));
    cudaFree(P->d_io);
  }
  P->d_io = nullptr;
  P->io_bytes = 0;
  PCUDA(P, cudaMalloc(&P->d_io, bytes));
  P->io_bytes = bytes;
  return GP_OK;
}

}  // namespace

// =================================================================== C ABI

extern "C" {

int gp_pool_slot_bytes(const gp_params* p, size_t* bytes) {
  size_t single = 0;
  if (!bytes) {
    gpk::set_thread_error("bytes is NULL");
    return GP_ERR_ARG;
  }
  const int rc = gp_workspace_bytes(p, &single);   // validates p
  if (rc != GP_OK) return rc;
  SlotGeom G;
  slot_geometry(*p, &G);
  *bytes = G.total;
  return GP_OK;
}

int gp_pool_create(size_t arena_bytes, int max_slots, void* stream, gp_pool** out) {
  if (!out) {
    gpk::set_thread_error("out is NULL");
    return GP_ERR_ARG;
  }
  *out = nullptr;
  if (arena_bytes == 0 || max_slots < 1 || max_slots > kMaxPoolSlots) {
    gpk::set_thread_error("arena_bytes must be > 0 and max_slots within 1..4096");
    return GP_ERR_ARG;
  }
  gp_pool* P = new gp_pool();
  auto bail = [&](int code, const std::string& msg) {
    gpk::set_thread_error(msg.c_str());
    gp_pool_destroy(P);
    return code;
  };
  cudaError_t e = cudaGetDevice(&P->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&P->nsm, cudaDevAttrMultiProcessorCount, P->device);
  if (e != cudaSuccess) return bail(GP_ERR_CUDA, std::string("device query: ") + cudaGetErrorString(e));
  if (stream) {
    P->stream = static_cast<cudaStream_t>(stream);
  } else {
    // the step is captured as a graph, which the legacy default stream does not allow
    e = cudaStreamCreateWithFlags(&P->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(GP_ERR_CUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e));
    P->owns_stream = true;
  }
  P->capacity = align_up(arena_bytes, kAlign);
  e = cudaMalloc(&P->arena, P->capacity);
  if (e != cudaSuccess) {
    cudaGetLastError();
    P->arena = nullptr;
    return bail(GP_ERR_NOMEM, std::string("cudaMalloc (arena): ") + cudaGetErrorString(e));
  }
  P->alloc.reset(P->capacity);
  P->slots.resize(max_slots);
  P->h_desc.resize(max_slots);
  const size_t part = (size_t)gpk::kReduceBlocks * gpk::kObsAcc * 8;
  const size_t scratch = part + 256;
  e = cudaMalloc(&P->d_desc, sizeof(SlotDesc) * max_slots);
  if (e == cudaSuccess) e = cudaMalloc(&P->d_scratch, scratch);
  if (e == cudaSuccess) e = cudaMemsetAsync(P->d_scratch, 0, scratch, P->stream);
  if (e != cudaSuccess) return bail(GP_ERR_NOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  P->d_partials = reinterpret_cast<double*>(P->d_scratch);
  P->d_counter = reinterpret_cast<unsigned int*>(P->d_scratch + part);
  P->d_obs = reinterpret_cast<double*>(P->d_scratch + part + 64);
  P->d_status = reinterpret_cast<int*>(P->d_scratch + part + 192);
  *out = P;
  return GP_OK;
}

void gp_pool_destroy(gp_pool* P) {
  if (!P) return;
  if (P->stream) cudaStreamSynchronize(P->stream);
  drop_graph(P);
  for (int m = 0; m < 2; ++m)
    for (int a = 0; a < 3; ++a)
      if (P->d_items[m][a]) cudaFree(P->d_items[m][a]);
  if (P->d_io) cudaFree(P->d_io);
  if (P->d_scratch) cudaFree(P->d_scratch);
  if (P->d_desc) cudaFree(P->d_desc);
  if (P->arena) cudaFree(P->arena);
  if (P->owns_stream) cudaStreamDestroy(P->stream);
  delete P;
}

int gp_pool_free_bytes(const gp_pool* P, size_t* free_bytes, size_t* largest) {
  if (!P || !free_bytes || !largest) return GP_ERR_ARG;
  *free_bytes = P->alloc.free_total();
  *largest = P->alloc.largest();
  return GP_OK;
}

int gp_pool_add(gp_pool* P, const gp_params* p, int* slot) {
  if (!P || !p || !slot) return P ? pfail(P, GP_ERR_ARG, "params or slot is NULL") : GP_ERR_ARG;
  *slot = -1;
  size_t single = 0;
  if (gp_workspace_bytes(p, &single) != GP_OK)
    return pfail(P, GP_ERR_ARG, gp_last_error(nullptr));
  if (p->prec != GP_F32) return pfail(P, GP_ERR_ARG, "pools hold FP32 fields (prec = GP_F32)");
  int idx = -1;
  for (int i = 0; i < (int)P->slots.size(); ++i)
    if (!P->slots[i].live) {
      idx = i;
      break;
    }
  if (idx < 0) return pfail(P, GP_ERR_NOMEM, "every slot of the pool is in use");
  Slot S;
  S.prm = *p;
  S.g = nonlinearity_of(*p);
  S.mode = 0;
  slot_geometry(*p, &S.G);
  std::vector<unsigned char> tabs;
  if (!slot_tables(*p, S.G, &S, &tabs))
    return pfail(P, GP_ERR_ARG,
                 "pools need every extent >= 8 and dt / h^2 small enough for a band of half-width <= 8");
  if (!P->alloc.alloc(S.G.total, &S.off)) return pfail(P, GP_ERR_NOMEM, "the arena has no free range large enough");
  S.live = true;
  P->slots[idx] = S;
  unsigned char* b = slot_base(P, P->slots[idx]);
  auto undo = [&](int code) {
    P->slots[idx].live = false;
    P->alloc.release(S.off, S.G.total);
    return code;
  };
  cudaError_t e = cudaMemcpyAsync(b + S.G.off_fx[0], tabs.data(), tabs.size(), cudaMemcpyHostToDevice, P->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(b + S.G.off_scal, 0, 64, P->stream);
  if (e != cudaSuccess) return undo(pcuda(P, e, "slot tables"));
  // the g = 0 trap ground state, normalised through the pending factor
  FieldParams f = slot_field(P, idx);
  f.out = reinterpret_cast<double*>(b + S.G.off_scal);
  e = gpk::launch_init_gaussian<float>(f, p->gamma, p->nu, p->lambda, P->stream);
  if (e == cudaSuccess) e = gpk::launch_norm_to_scale<float>(f, P->stream);
  if (e != cudaSuccess) return undo(pcuda(P, e, "slot init"));
  // tables are staged in host memory: finish the copy before `tabs` goes away
  e = cudaStreamSynchronize(P->stream);
  if (e != cudaSuccess) return undo(pcuda(P, e, "slot init"));
  P->dirty = true;
  *slot = idx;
  return GP_OK;
}

int gp_pool_remove(gp_pool* P, int slot) {
  if (!slot_ok(P, slot)) return P ? pfail(P, GP_ERR_ARG, "no such live slot") : GP_ERR_ARG;
  PCUDA(P, cudaStreamSynchronize(P->stream));
  Slot& S = P->slots[slot];
  P->alloc.release(S.off, S.G.total);
  S.live = false;
  P->dirty = true;
  return GP_OK;
}

int gp_pool_set_real_time(gp_pool* P, int slot) {
  if (!slot_ok(P, slot)) return P ? pfail(P, GP_ERR_ARG, "no such live slot") : GP_ERR_ARG;
  Slot& S = P->slots[slot];
  if (S.mode == 1) return GP_OK;
  unsigned char* b = slot_base(P, S);
  const long long rows = (long long)S.prm.ny * S.prm.nz;
  double* scale = reinterpret_cast<double*>(b + S.G.off_scal);
  k_real_to_complex<<<(unsigned int)std::min<long long>(rows, 4096), 256, 0, P->stream>>>(
      reinterpret_cast<const float*>(b + S.G.off_field), S.G.pitch[0],
      reinterpret_cast<float2*>(b + S.G.off_staging), S.G.pitch[1], S.prm.nx, rows, scale);
  PCUDA(P, cudaGetLastError());
  PCUDA(P, cudaMemcpyAsync(b + S.G.off_field, b + S.G.off_staging, (size_t)S.G.pitch[1] * 8 * rows,
                           cudaMemcpyDeviceToDevice, P->stream));
  k_pool_set_double<<<1, 1, 0, P->stream>>>(scale, 1.0);
  PCUDA(P, cudaGetLastError());
  S.mode = 1;
  P->dirty = true;
  return GP_OK;
}

int gp_pool_set_g(gp_pool* P, int slot, double g) {
  if (!slot_ok(P, slot) || !std::isfinite(g)) return P ? pfail(P, GP_ERR_ARG, "no such live slot or g not finite") : GP_ERR_ARG;
  P->slots[slot].g = g;
  if (!P->dirty) {   // descriptors are read from device memory: no new graph needed
    P->h_desc[slot].dtg = (float)(P->slots[slot].prm.dt * g);
    PCUDA(P, cudaMemcpyAsync(P->d_desc + slot, &P->h_desc[slot], sizeof(SlotDesc),
                             cudaMemcpyHostToDevice, P->stream));
    PCUDA(P, cudaStreamSynchronize(P->stream));
  }
  return GP_OK;
}

int gp_pool_step(gp_pool* P, long nsteps) {
  if (!P || nsteps < 0) return P ? pfail(P, GP_ERR_ARG, "nsteps must be >= 0") : GP_ERR_ARG;
  const int rc = run_steps(P, nsteps);
  if (rc != GP_OK) return rc;
  return check_status(P);
}

int gp_pool_observables(gp_pool* P, int slot, gp_obs* out) {
  if (!slot_ok(P, slot) || !out) return P ? pfail(P, GP_ERR_ARG, "no such live slot or out is NULL") : GP_ERR_ARG;
  const FieldParams f = slot_field(P, slot);
  cudaError_t e = gpk::launch_observables<float>(f, P->slots[slot].mode == 1, P->stream);
  if (e != cudaSuccess) return pcuda(P, e, "observables");
  double o[10];
  PCUDA(P, cudaMemcpyAsync(o, P->d_obs, sizeof o, cudaMemcpyDeviceToHost, P->stream));
  const int rc = check_status(P);
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

int gp_pool_get_psi(gp_pool* P, int slot, double* host, int as_complex) {
  if (!slot_ok(P, slot) || !host || (as_complex != 0 && as_complex != 1))
    return P ? pfail(P, GP_ERR_ARG, "bad arguments") : GP_ERR_ARG;
  const Slot& S = P->slots[slot];
  if (S.mode == 1 && !as_complex) return pfail(P, GP_ERR_STATE, "the field is complex; request it with as_complex = 1");
  const size_t N = (size_t)S.prm.nx * S.prm.ny * S.prm.nz;
  int rc = ensure_io(P, N * 16);
  if (rc != GP_OK) return rc;
  const FieldParams f = slot_field(P, slot);
  cudaError_t e = gpk::launch_export<float>(f, P->d_io, S.mode == 1, as_complex == 1, P->stream);
  if (e != cudaSuccess) return pcuda(P, e, "export");
  PCUDA(P, cudaMemcpyAsync(host, P->d_io, N * 8 * (as_complex ? 2 : 1), cudaMemcpyDeviceToHost, P->stream));
  return check_status(P);
}

int gp_pool_set_psi(gp_pool* P, int slot, const double* host, int is_complex) {
  if (!slot_ok(P, slot) || !host || (is_complex != 0 && is_complex != 1))
    return P ? pfail(P, GP_ERR_ARG, "bad arguments") : GP_ERR_ARG;
  Slot& S = P->slots[slot];
  const size_t N = (size_t)S.prm.nx * S.prm.ny * S.prm.nz;
  int rc = ensure_io(P, N * 16);
  if (rc != GP_OK) return rc;
  PCUDA(P, cudaMemcpyAsync(P->d_io, host, N * 8 * (is_complex ? 2 : 1), cudaMemcpyHostToDevice, P->stream));
  if (S.mode != is_complex) P->dirty = true;
  S.mode = is_complex;
  const FieldParams f = slot_field(P, slot);
  cudaError_t e = gpk::launch_import<float>(f, P->d_io, is_complex == 1, P->stream);
  if (e != cudaSuccess) return pcuda(P, e, "import");
  k_pool_set_double<<<1, 1, 0, P->stream>>>(reinterpret_cast<double*>(slot_base(P, S) + S.G.off_scal), 1.0);
  PCUDA(P, cudaGetLastError());
  PCUDA(P, cudaStreamSynchronize(P->stream));
  return GP_OK;
}

int gp_pool_set_graph(gp_pool* P, int enable) {
  if (!P || (enable != 0 && enable != 1)) return P ? pfail(P, GP_ERR_ARG, "enable must be 0 or 1") : GP_ERR_ARG;
  P->use_graph = enable == 1;
  drop_graph(P);
  return GP_OK;
}

int gp_pool_set_shape(gp_pool* P, int x_stages, int seg_turns) {
  if (!P || x_stages < 2 || x_stages > 8 || seg_turns < 1 || seg_turns > 8)
    return P ? pfail(P, GP_ERR_ARG, "x_stages within 2..8 and seg_turns within 1..8") : GP_ERR_ARG;
  P->x_stages = x_stages;
  P->seg_turns = seg_turns;
  P->dirty = true;
  return GP_OK;
}

int gp_pool_tune(gp_pool* P, int steps_per_candidate, double* best_ms) {
  if (!P || steps_per_candidate < 1) return P ? pfail(P, GP_ERR_ARG, "steps_per_candidate must be >= 1") : GP_ERR_ARG;
  const size_t hw = P->alloc.high_water();
  if (hw == 0) return pfail(P, GP_ERR_STATE, "no live slot to tune on");
  PCUDA(P, cudaStreamSynchronize(P->stream));
  void* snap = nullptr;
  PCUDA(P, cudaMalloc(&snap, hw));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int stages[3] = {2, 3, 4}, turns[4] = {1, 2, 3, 4};
  int best_s = P->x_stages, best_t = P->seg_turns;
  float best = 1e30f;
  int rc = GP_OK;
  cudaError_t ce = cudaMemcpyAsync(snap, P->arena, hw, cudaMemcpyDeviceToDevice, P->stream);
  if (ce != cudaSuccess) rc = pcuda(P, ce, "tune snapshot");
  for (int si = 0; si < 3 && rc == GP_OK; ++si)
    for (int ti = 0; ti < 4 && rc == GP_OK; ++ti) {
      P->x_stages = stages[si];
      P->seg_turns = turns[ti];
      P->dirty = true;
      rc = run_steps(P, 1);   // builds lists and graph, warms up
      if (rc != GP_OK) break;
      cudaEventRecord(e0, P->stream);
      rc = run_steps(P, steps_per_candidate);
      cudaEventRecord(e1, P->stream);
      if (rc == GP_OK) rc = check_status(P);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rc == GP_OK && ms < best) {
        best = ms;
        best_s = stages[si];
        best_t = turns[ti];
      }
      ce = cudaMemcpyAsync(P->arena, snap, hw, cudaMemcpyDeviceToDevice, P->stream);
      if (ce != cudaSuccess && rc == GP_OK) rc = pcuda(P, ce, "tune restore");
    }
  cudaStreamSynchronize(P->stream);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(snap);
  P->x_stages = best_s;
  P->seg_turns = best_t;
  P->dirty = true;
  if (best_ms) *best_ms = best < 1e30f ? best / steps_per_candidate : -1.0;
  return rc;
}

int gp_pool_info(const gp_pool* P, long long info[8]) {
  if (!P || !info) return GP_ERR_ARG;
  long long live = 0;
  for (const auto& S : P->slots) live += S.live ? 1 : 0;
  info[0] = live;
  info[1] = (long long)(P->capacity - P->alloc.free_total());
  info[2] = P->x_stages;
  info[3] = P->seg_turns;
  info[4] = (P->exec ? 1 : 0) | (P->x_reg[0] ? 2 : 0) | (P->x_reg[1] ? 4 : 0);
  info[5] = P->launches_per_step;
  info[6] = (long long)P->alloc.free_total();
  info[7] = (long long)P->alloc.largest();
  return GP_OK;
}

const char* gp_pool_last_error(const gp_pool* P) { return P ? P->err.c_str() : gp_last_error(nullptr); }

}  // extern "C"

// gp_internal.h -- declarations shared by the host runtime (gp_api.cu) and the
// kernel translation units (gp_sweeps.cu, gp_reduce.cu).  Not part of the ABI.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <complex>
#include <vector>

namespace gpk {

// Status bits written by kernels into the solver's device status word.
constexpr int kStatusNonFinite = 1;  // norm non-finite or zero (imaginary time)
constexpr int kStatusTimeout = 2;    // a bounded wait on a tile copy ran out
constexpr int kStatusBounds = 4;     // GP_CHECK builds: an index fell outside its buffer

// Bounded waits on a block's own copies give up after this much wall time.  A
// solver's first wait on each copy takes its own limit (SweepParams::wait_ns, this
// value unless gp_set_wait_limit changed it); the wait that drains the copies still
// in flight after a timeout always takes this one, so that no copy is left writing
// into shared memory after the block exits.
constexpr uint64_t kWaitLimitNs = 2000000000ull;

// Largest grid extent per axis accepted by the ABI.
constexpr int kMaxExtent = 2048;
// Longest line segment one TMA box covers (hardware limit on a box dimension).
constexpr int kMaxBox = 256;

// Warps per block of the banded FP32 x sweep (each warp works on its own rows): few
// large blocks fill the SMs sooner than many small ones when the sweep starts.
constexpr int kBandWarps = 12;
// Warps per block of the register-row banded x sweep (each warp on its own rows).
constexpr int kXRegWarps = 8;
// Warps per block of the batched x sweep (one work item per warp).
constexpr int kBatchXWarps = 4;
// Largest half-width of the banded operators (weights arrays hold 2 kBandHalfMax + 1).
constexpr int kBandHalfMax = 8;

// Most warps per block of any kernel that ends with a block-level norm reduction (the
// per-warp arrays of those reductions are sized by it; their blocks have 4 to 12
// warps).  Small static arrays matter: the banded y / z blocks take 45 KB of dynamic
// shared memory each, five to an SM, with little room to spare.
constexpr int kMaxBlockWarps = 16;

// Ticket counters of the fused norm: a solver's counters[0] is the top counter,
// counters[kNormGroupBase .. + kNormGroups) the group counters (the solver's scalar
// area holds 48 counters).
constexpr int kNormGroups = 32;
constexpr int kNormGroupBase = 16;

// Fixed launch shape of the reductions, so that their summation order (and hence
// their result) does not depend on the device.
constexpr int kReduceBlocks = 608;
constexpr int kReduceThreads = 256;

// Number of FP64 accumulators of the observables pass:
// 0 sum|psi|^2, 1 sum V|psi|^2, 2 sum|psi|^4, 3..5 edge sums along x, y, z,
// 6..8 sum x^2|psi|^2, y^2.., z^2..
constexpr int kObsAcc = 9;

// Arguments of one sweep launch.  Coefficient arrays hold R (real field) or the
// complex pair of R (complex field):
//   A_j = m_j (1 - 2a),  B_j = a m_j,  with m_j the Thomas pivots (see gp_api.cu).
struct SweepParams {
  void* psi;             // field read by the sweep, layout [nz][ny][pitch]
  void* out;             // field written (== psi except for the FP32 y / z sweeps)
  int nx, ny, nz;
  int pitch;             // row pitch of the field in elements
  int n;                 // line length along the swept axis
  int lines;             // lines per tile (one lane per line)
  int tiles_x;           // x-tiles per (j or k) for the y / z sweeps
  int box;               // TMA box length along the swept axis
  int nbox;              // boxes per line
  int words_per_elem;    // 1 real, 2 complex (TMA coordinates are in words)
  const void* A;
  const void* B;
  int head;              // coefficients j >= head equal entry n-1 exactly (in storage precision)
  int trunc;             // FP32 fast sweeps: truncation depth L of the decaying coupling
  int nseg;              // FP32 fast y / z sweeps: segments per line
  // FP32 banded x sweep (band_w > 0)
  const void* band_fx;   // trap factors along x: exp(-dt V_x) or cis(-dt V_x), [pitch], FP32
  const void* band_fyz;  // trap factor per row r = k ny + j: exp(-dt (V_y + V_z)) or cis(..)
  float band_wt[2 * 17]; // free-line CN row w_{k - band_w}, k = 0 .. 2 band_w, centre as w_0 - 1 (complex: pairs)
  int band_w;            // half-width W of the band (3, 5 or 8)
  int band_rows;         // x: consecutive rows per warp; the first band_rem warps take one more
  int band_rem;
  int band_stages;       // x: groups of rows in flight per warp
  int band_group;        // x: rows per group (worked on together by the warp's lanes)
  int band_seg;          // y / z: points per line segment (a multiple of 2 band_w + 1)
  int band_cp;           // y / z: 1 = next turn's inputs copied to shared memory ahead (cp.async)
  int band_reg;          // x: 1 = the row in registers (k_sweep_x_reg)
  float band_dtg;        // x: dt g in FP32
  // pointwise substep (x sweep only)
  int pw;                // 1: pointwise substep fused on load; 0: kinetic-only step
  const void* vx;
  const void* vy;
  const void* vz;
  double dt, g;
  const double* scale;   // pending renormalisation factor, applied on load
  // fused norm (z sweep, imaginary time only)
  double* partials;
  unsigned int* counter;
  double* scale_out;
  // deferred finish of the fused norm (FP32 real field): the z sweep stores its
  // per-block partials (norm_blocks of them) and sets *scale_state = 1; the next x
  // sweep (every block, the same fixed order) sums them into the factor it applies,
  // and any other reader of the factor first runs k_resolve_scale
  int norm_defer;        // z: store partials only; x: take the factor from the partials
  int norm_blocks;       // blocks of the z sweep (partials to sum)
  int norm_copies;       // z stores norm_copies copies of its partials (copy c at c norm_blocks);
                         // x block b reads copy b mod norm_copies: fewer readers per L2 line
  int* scale_state;      // 1: the factor is the partials' 1 / sqrt(sum dV)
  // FP32 field in imaginary time: the step counter behind the renormalisation factor's
  // dither (step_dither in gp_device.cuh): the sweeps that apply the factor read it, the
  // y sweep adds one; null otherwise (no dither)
  unsigned int* step_ctr;
  int* status;
  double dV;
  long long ntiles;
  unsigned long long wait_ns;   // limit of the first bounded wait on each copy
};

// One resident solve of a pool (gp_batch.cu), as the batched FP32 sweeps see it.
struct SlotDesc {
  void* field;            // [nz][ny][pitch] elements (float or complex pairs)
  void* staging;          // same layout: the y sweep writes it, the z sweep reads it
  const void* fx;         // trap factors along x, [pitch]
  const void* fyz;        // trap factor per row r = k ny + j
  double* scale;          // pending renormalisation factor (imaginary time)
  double* partials;       // z-sweep norm partials, one per z block of the slot
  unsigned int* counter;  // z blocks of the slot finished (reset by the last)
  int nx, ny, nz, pitch;
  int seg[3];             // y / z: segment length in points
  float dtg;              // dt g
  double dV;
  // banded weights per axis, w_{k-8}, k = 0 .. 16 (centre as w_0 - 1; complex:
  // pairs), zero beyond the slot's own half-width
  float wt[3][2 * (2 * kBandHalfMax + 1)];
};
// One warp's rows of a batched x sweep.
struct XItem {
  int slot;
  int nrow;
  long long row0;
  int group;              // rows per group (<= BatchArgs::group_max)
  int pad;
};
// One block of a batched y / z sweep: block blk of the nblk blocks of one slot.
struct LineBlock {
  int slot;
  int blk;
  int nblk;
  int pad;
};
// Arguments of a batched sweep launch.
struct BatchArgs {
  const SlotDesc* slots;
  const void* items;      // XItem (x) or LineBlock (y, z), one per warp / block
  int nitems;
  int stages;             // x: groups of rows in flight per warp
  int group_max;          // x: row slots per stage (the largest group of the items)
  int slot_elems;         // x: shared-memory row slot, elements (>= pitch + 16 of every slot)
  int* status;
  unsigned long long wait_ns;   // limit of the first bounded wait on each copy
  int x_reg;              // x: rows in registers (k_batch_x_reg), items of `group` rows per pass
};

// Arguments of the reductions and conversion kernels.
struct FieldParams {
  void* psi;
  int nx, ny, nz, pitch;
  const double* scale;
  double* partials;
  unsigned int* counter;
  double* out;           // result (observables: 10 values; norm: the scale)
  int* status;
  const double* tab;     // FP64 tables: V_x[nx] V_y[ny] V_z[nz] x^2[nx] y^2[ny] z^2[nz]
  double hx, hy, hz, g;
};

// Kernel launchers (gp_sweeps.cu / gp_reduce.cu).  R = double or float storage.
template <class R> cudaError_t launch_sweep_x(const SweepParams& p, bool complex_field,
                                              size_t smem, cudaStream_t st);
template <class R> cudaError_t launch_sweep_y(const CUtensorMap& map, const SweepParams& p,
                                              bool complex_field, size_t smem, cudaStream_t st);
template <class R> cudaError_t launch_sweep_z(const CUtensorMap& map, const SweepParams& p,
                                              bool complex_field, size_t smem, cudaStream_t st);
template <class R> cudaError_t sweep_set_smem_limits(size_t max_smem);
// FP32 shared-memory-free sweeps (x: streaming, one lane per row, 32 rows per warp;
// y, z: streaming, one lane per line); y / z grid in blocks of 128 threads.
cudaError_t launch_sweep_fast(int axis, const SweepParams& p, bool complex_field, int grid,
                              cudaStream_t st);
// FP32 banded x sweep: dynamic shared memory of a block of kBandWarps warps, one-time
// preparation (shared-memory limit, resident blocks per SM) and launch on `grid` blocks.
size_t x_band_smem(const SweepParams& p, bool complex_field);
cudaError_t x_band_prepare(int w, bool complex_field, bool grouped, size_t smem,
                           int* blocks_per_sm);
cudaError_t launch_sweep_x_band(const SweepParams& p, bool complex_field, int grid,
                                cudaStream_t st);
// FP32 banded x sweep with the row in registers (rows of nx = 8 m <= 256, W in {3, 5}):
// blocks of kXRegWarps warps, no shared memory; band_rows rows per warp.
bool x_reg_fits(int nx, int w);
cudaError_t x_reg_prepare(int w, bool complex_field, int* blocks_per_sm);
cudaError_t launch_sweep_x_reg(const SweepParams& p, bool complex_field, int grid, cudaStream_t st);
// FP32 banded y / z sweeps (out of place like the streaming ones), blocks of 128 threads.
cudaError_t launch_sweep_band_line(int axis, const SweepParams& p, bool complex_field, int grid,
                                   cudaStream_t st);
int band_line_blocks_per_sm(int axis, bool complex_field, int w, bool cp);
// Batched FP32 banded sweeps over the slots of a pool (one launch per direction
// and mode): x on kBandWarps-warp blocks with dynamic shared memory
// batch_x_smem(); y / z on blocks of 128 threads.  w is the launch half-width.
size_t batch_x_smem(int stages, int group_max, int slot_elems, bool complex_field);
// Rows per group of the banded x sweep for rows of nx points (ept per 16-byte vector):
// the cost model's best G in 1..8 whose stages fit warp_budget bytes of row slots.
int x_band_group(int nx, int ept, int stages, size_t slot_bytes, size_t warp_budget);
cudaError_t batch_prepare(int w, bool complex_field, size_t x_smem, int* x_blocks_per_sm);
cudaError_t launch_batch_sweep(int axis, int w, const BatchArgs& b, bool complex_field, int grid,
                               size_t smem, cudaStream_t st);
// Batched x sweep with rows in registers (slots of nx = 16 m <= 512 real or 8 m <= 256
// complex points, W in {3, 5}): whether a slot fits, and the resident blocks of
// kXRegWarps warps per SM.
bool batch_x_reg_fits(int nx, int w, bool complex_field);
cudaError_t batch_x_reg_prepare(int w, bool complex_field, int* blocks_per_sm);
// FP64 sweeps (gp_sweeps64.cu): x moves 32 rows per warp through shared-memory
// chunks (dynamic shared memory x64_smem), y / z stream one line per thread; the
// launch covers the whole grid (sweep64_blocks blocks).  sweep64_prepare sets the x
// kernels' shared-memory limit (once per device).
size_t x64_smem(bool complex_field);
cudaError_t sweep64_prepare();
long long sweep64_blocks(int axis, int nx, int ny, int nz);
cudaError_t launch_sweep64(int axis, const SweepParams& p, bool complex_field, cudaStream_t st);
// Resident warps per SM of the streaming y / z kernel (occupancy calculator).
int stream_warps_per_sm(int axis, bool complex_field, int trunc);

template <class R> cudaError_t launch_observables(const FieldParams& p, bool complex_field,
                                                  cudaStream_t st);
// Standalone pointwise substep over the field (Strang splitting's half steps): trap
// factors fx [pitch] and fyz [rows] of the half step, dtg = (dt / 2) g; the pending
// factor *p.scale applied first when apply_scale; with norm, *p.out receives
// 1 / sqrt(sum |psi|^2 dV) of the result (fixed-order FP64 sum).
template <class R> cudaError_t launch_half_pointwise(const FieldParams& p, bool complex_field,
                                                     const void* fx, const void* fyz, double dtg,
                                                     bool apply_scale, bool norm, cudaStream_t st);
template <class R> cudaError_t launch_norm_to_scale(const FieldParams& p, cudaStream_t st);
// When *state is 1: the factor 1 / sqrt(dV sum of the nb float-float partials) into
// *scale (non-finite or zero norm flagged in *status), and *state = 0 (one block).
cudaError_t launch_resolve_scale(double* scale, int* state, const double* partials, int nb,
                                 double dV, int* status, cudaStream_t st);
// FP32 field times *p.scale, packed into rows of nx elements in dst (not aliasing the
// field); the field and the factor are left as they are.
cudaError_t launch_export_f32(const FieldParams& p, bool complex_field, float* dst, cudaStream_t st);
// Packed rows of nx FP32 elements (real or complex pairs) from src into the field,
// pad columns zero.
cudaError_t launch_import_f32(const FieldParams& p, bool complex_field, const float* src, cudaStream_t st);
template <class R> cudaError_t launch_init_gaussian(const FieldParams& p, double wx, double wy,
                                                    double wz, cudaStream_t st);
template <class R> cudaError_t launch_import(const FieldParams& p, const double* src,
                                             bool complex_field, cudaStream_t st);
template <class R> cudaError_t launch_export(const FieldParams& p, double* dst,
                                             bool complex_field, bool as_complex, cudaStream_t st);
template <class R> cudaError_t launch_density2d(const FieldParams& p, bool complex_field,
                                                int plane, double* out, cudaStream_t st);
cudaError_t launch_rows_sum(const double* in, int rows, int cols, double w, double* out,
                            cudaStream_t st);
cudaError_t launch_cols_sum(const double* in, int rows, int cols, double w, double* out,
                            cudaStream_t st);

// Message returned by gp_last_error(NULL) on this thread (gp_api.cu).
void set_thread_error(const char* msg);

// Row of the free-line CN operator for a = tau / (4 h^2) (gp_api.cu): returns the
// half-width W in {3, 5, 8} that keeps the neglected entries below 2^-28 and the
// weights w[0 .. 2W] (w[W] the centre), or 0.
int cn_free_row(std::complex<double> a, std::vector<std::complex<double>>* w);

}  // namespace gpk

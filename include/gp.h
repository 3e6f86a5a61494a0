/*
 * gp.h -- C ABI of the GB300 (sm_103a) split-step Crank-Nicolson solver for the
 * time-dependent Gross-Pitaevskii (GP) equation in a fully anisotropic 3D
 * harmonic trap.
 *
 * Paper: "OpenMP Fortran and C programs for solving the time-dependent
 * Gross-Pitaevskii equation in an anisotropic trap", program summary:
 *   - Nature of problem: GP equation for a condensate with contact interaction in a
 *     fully anisotropic 3D harmonic trap.
 *   - Solution method: split-step Crank-Nicolson (SSCN) discretisation in space and
 *     time, propagation over small steps in imaginary time (stationary state) or
 *     real time (dynamics).
 *   - Summary of revisions: inputs are the number of atoms, the scattering length
 *     and the oscillator length, from which the dimensionless nonlinearity is
 *     computed; outputs are energy, chemical potential, rms sizes, the density and
 *     the integrated 1D / 2D densities (Eq. 1); the real-time run starts from the
 *     imaginary-time state and multiplies the nonlinearity by a factor (quench).
 *
 * Equation and discretisation (the paper names the method but prints neither; the
 * textbook forms are used):
 *   i dpsi/dt = [-(1/2) Lap + V + g |psi|^2] psi,
 *   V = (gamma^2 x^2 + nu^2 y^2 + lambda^2 z^2) / 2,   g = 4 pi N a_s / l_osc.
 *   Grid x_i = (i - (nx-1)/2) dx, i = 0..nx-1 (box centred on the origin), same for
 *   y and z; psi = 0 on the ghost points just outside the box.
 *   One step, tau = dt (imaginary time, real field) or i dt (real time, complex field):
 *     1. psi <- psi exp(-tau (V + g |psi|^2))                     (pointwise)
 *     2. per axis x, y, z, on every grid line, one Crank-Nicolson solve
 *        (1+2a) u_j - a (u_{j-1}+u_{j+1}) = (1-2a) v_j + a (v_{j-1}+v_{j+1}),
 *        a = tau / (4 h^2), by a Thomas recurrence with precomputed coefficients
 *     3. imaginary time: psi <- psi / sqrt(sum |psi|^2 dV)           (renormalise)
 *
 * Conventions for every call:
 *   - Return 0 on success or a negative GP_ERR_* code; nothing is thrown.
 *   - Host pointers are owned by the caller and are only used during the call.
 *   - Device memory is owned by the library (gp_create) or by the caller
 *     (gp_create_on); the solver never frees a caller's buffer.
 *   - Work is queued on the stream given at creation (NULL: the legacy default
 *     stream).  gp_step_* return as soon as the work is queued; gp_sync,
 *     gp_observables, gp_get_psi and the density calls wait for it, and report
 *     GP_ERR_NONFINITE when a step produced a non-finite or zero norm and
 *     GP_ERR_TIMEOUT when a kernel's bounded wait on its own copies ran out (and,
 *     in a library built with -DGP_CHECK, GP_ERR_BOUNDS when a kernel's bounds
 *     check found an index outside its buffer: the access is skipped, nothing traps).
 *   - Host-side arrays use the layout psi[k][j][i] (x fastest, index
 *     (k*ny + j)*nx + i), FP64, complex values interleaved (re, im), whatever the
 *     storage precision on the device.
 *   - A solver is not thread-safe; distinct solvers are independent.
 */
#ifndef GP_H
#define GP_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GP_OK 0
#define GP_ERR_ARG (-1)       /* invalid argument or unsupported size          */
#define GP_ERR_NOMEM (-2)     /* device allocation failed or buffer too small  */
#define GP_ERR_CUDA (-3)      /* a CUDA call failed (see gp_last_error)        */
#define GP_ERR_NONFINITE (-4) /* the norm became non-finite or zero            */
#define GP_ERR_TIMEOUT (-5)   /* a kernel's bounded wait gave up               */
#define GP_ERR_STATE (-6)     /* call not valid in the solver's current mode   */
#define GP_ERR_BOUNDS (-7)    /* a bounds check of a GP_CHECK build failed     */

/* Storage precision of the field.  FP64: double / complex double, all arithmetic
 * in FP64.  FP32: float / complex float storage and sweeps; elimination
 * coefficients computed in FP64 and rounded once; norm and observables
 * accumulated in FP64.                                                           */
typedef enum { GP_F64 = 0, GP_F32 = 1 } gp_prec;

/* Problem definition ("Summary of revisions": physical inputs, trap anisotropy).
 *   nx, ny, nz     grid points per axis, each 3..2048; nz = 1 makes a 2D solve in
 *                  the xy plane (the imag2d / real2d programs): z = 0, no z solve,
 *                  cell area dx dy in every sum, g the 2D nonlinearity, dz and lambda
 *                  unused; rms_z is then 0
 *   dx, dy, dz     grid spacings (> 0), dimensionless (units of the x oscillator length)
 *   dt             time step (> 0)
 *   gamma, nu, lambda  trap frequencies relative to the x trap (> 0)
 *   use_physical   0: take g as given; 1: g = 4 pi natoms a_s / l_osc, with a_s and
 *                  l_osc in the same length unit
 *   prec           gp_prec                                                       */
typedef struct {
  int nx, ny, nz;
  double dx, dy, dz;
  double dt;
  double gamma, nu, lambda;
  int use_physical;
  double g;
  double natoms, a_s, l_osc;
  int prec;
} gp_params;

/* Observables ("Summary of revisions": energy, chemical potential, rms sizes).
 *   norm   = sum |psi|^2 dV
 *   ekin   = <psi| -(1/2) Lap_h |psi> dV   (3-point Laplacian, zero ghosts: the
 *            operator of the CN substep)
 *   epot   = sum V |psi|^2 dV,   eint = (g/2) sum |psi|^4 dV
 *   energy = ekin + epot + eint,  mu = ekin + epot + 2 eint
 *   rms_a  = sqrt(sum a^2 |psi|^2 dV / norm), rms_r = sqrt(rms_x^2+rms_y^2+rms_z^2)
 * energy and mu are the per-atom values for a unit-norm state, which imaginary
 * time enforces and real time conserves.                                         */
typedef struct {
  double norm, mu, energy, ekin, epot, eint, rms_x, rms_y, rms_z, rms_r;
} gp_obs;

typedef struct gp_solver gp_solver;

/* Device bytes that gp_create_on needs for these parameters (host only, no CUDA
 * call).  Returns GP_ERR_ARG for invalid parameters.                             */
int gp_workspace_bytes(const gp_params* p, size_t* bytes);

/* Validate p, compute g, the Crank-Nicolson elimination coefficients (FP64) and
 * the trap tables, allocate the device state with cudaMalloc on the current
 * device and bind `stream` (a cudaStream_t, or NULL).  The field starts at zero.
 * *out receives the solver, or NULL on error (then gp_last_error(NULL) explains). */
int gp_create(const gp_params* p, void* stream, gp_solver** out);

/* Same, inside a caller-owned device buffer of `bytes` >= gp_workspace_bytes,
 * 256-byte aligned, that must outlive the solver.                                */
int gp_create_on(const gp_params* p, void* dev_buf, size_t bytes, void* stream,
                 gp_solver** out);

/* Wait for queued work, free library-owned memory and the solver.  NULL is a no-op. */
void gp_destroy(gp_solver* s);

/* Real field exp(-(wx x^2 + wy y^2 + wz z^2) / 2) normalised on the grid; with
 * (wx, wy, wz) = (gamma, nu, lambda) it is the g = 0 trap ground state.
 * Puts the solver in imaginary-time (real field) mode.                           */
int gp_init_gaussian(gp_solver* s, double wx, double wy, double wz);

/* Copy a host field in (nx*ny*nz doubles, or 2*nx*ny*nz interleaved when
 * is_complex) and set the mode to real field / complex field accordingly.  The
 * field is taken as given (not renormalised).                                    */
int gp_set_psi(gp_solver* s, const double* host, int is_complex);

/* Copy the current (normalised) field out.  as_complex = 1 always works (a real
 * field gets zero imaginary parts); as_complex = 0 on a complex field returns
 * GP_ERR_STATE.  Synchronises.                                                   */
int gp_get_psi(gp_solver* s, double* host, int as_complex);

/* FP32 host I/O for FP32 solvers (prec GP_F32): as gp_set_psi / gp_get_psi with
 * float host buffers (nx*ny*nz floats, or 2*nx*ny*nz interleaved), one contiguous
 * host copy each way with no FP64 conversion (rows are re-pitched on the device when
 * the field's row pitch exceeds nx).
 * gp_get_psi_f32 returns the field times the pending renormalisation factor (packed
 * on the device in the solver's staging area; the solver's state is left as it is, so
 * a read does not change the bits of later steps).  as_complex must match the field
 * (0: real, 1: complex), else GP_ERR_STATE; FP64 solvers return GP_ERR_ARG.
 * gp_get_psi_f32 synchronises.                                                      */
int gp_set_psi_f32(gp_solver* s, const float* host, int is_complex);
int gp_get_psi_f32(gp_solver* s, float* host, int as_complex);

/* Overlapped read of an FP32 solver's field into host (same layout as
 * gp_get_psi_f32).  The field times the pending renormalisation factor is packed on
 * the device into one of two snapshot buffers of the solver, taken in turn (16 bytes
 * per grid point in all, cudaMalloc'd on the first call and freed by gp_destroy; the
 * solver's state is left as it is), and the device-to-host copy of the snapshot runs
 * on the solver's own copy stream: it overlaps whatever the caller enqueues next —
 * the next write (gp_set_psi_f32_async's host-to-device copy runs in the other
 * direction at the same time), the next steps and the next read's packing.  A read
 * waits, before it packs, for the copy of the read two before it (same buffer);
 * gp_sync(s) waits for all of them, and so do the synchronous reads, observables and
 * densities.  host is complete only after gp_sync(s) (or gp_destroy); it should be
 * page-locked for the copy to be asynchronous.  Does not read the status flag
 * (gp_sync does).  Same argument errors as gp_get_psi_f32; GP_ERR_NOMEM if the
 * snapshot buffers cannot be allocated, GP_ERR_CUDA if the copy stream cannot be
 * created.                                                                          */
int gp_get_psi_f32_async(gp_solver* s, float* host, int as_complex);

/* Overlapped write of an FP32 solver's field from host (same layout and arguments as
 * gp_set_psi_f32).  The host-to-device copy runs on the solver's own put stream into
 * one of two buffers of the solver, taken in turn (16 bytes per grid point in all,
 * cudaMalloc'd on the first call and freed by gp_destroy), beside whatever the solver
 * stream is doing (the steps and the packing of an overlapped read of the previous
 * field); the next call that reads or
 * writes the field (steps, reads, observables, densities, gp_sync, another write)
 * first waits for that copy and moves the buffer into the field on the solver stream,
 * with the effect of gp_set_psi_f32 (factor 1, step count 0).  host (page-locked for
 * the copy to overlap) must stay unchanged until a synchronising call (gp_sync, a
 * synchronous read, gp_observables, a density) has returned.  Same argument errors as
 * gp_set_psi_f32; GP_ERR_NOMEM if the buffer cannot be allocated, GP_ERR_CUDA if the
 * put stream cannot be created.                                                     */
int gp_set_psi_f32_async(gp_solver* s, const float* host, int is_complex);

/* nsteps imaginary-time SSCN steps on the real field, each renormalised to unit
 * norm.  GP_ERR_STATE on a complex field.  Asynchronous.  A call of one step
 * replays a CUDA graph of the step's launches, captured on the first such call (per
 * mode and splitting) on a stream of the solver's own; while the caller captures the
 * solver's stream, or if the capture fails, the step is launched directly.        */
int gp_step_imag(gp_solver* s, long nsteps);

/* nsteps real-time SSCN steps on the complex field.  On a real field the field is
 * first promoted to complex (imaginary parts zero): the imaginary-to-real-time
 * hand-off of the paper's real-time programs.  Asynchronous.  A call of one step
 * replays the step's CUDA graph as gp_step_imag does.                            */
int gp_step_real(gp_solver* s, long nsteps);

/* Replace the nonlinearity g (the paper's quench: the real-time run multiplies g
 * by a factor).  Takes effect for the next step.                                 */
int gp_set_g(gp_solver* s, double g);

/* Splitting of one time step.  GP_SPLIT_LIE (default): the pointwise substep with the
 * full dt, then the CN solves along x, y, z (one fused pass per axis).
 * GP_SPLIT_STRANG: half pointwise substep, CN solves, half pointwise substep, each
 * half taking |psi|^2 before its own update (second order in dt for the linear
 * part, and time-reversible in real time).  In real time n Strang steps cost n Lie
 * steps plus two pointwise passes (the inner halves merge exactly, the phase keeping
 * |psi|); in imaginary time each step adds two pointwise passes and renormalises
 * after the second.  Takes effect at the next step call.                          */
enum { GP_SPLIT_LIE = 0, GP_SPLIT_STRANG = 1 };
int gp_set_splitting(gp_solver* s, int scheme);

/* Current g (after the physical-units conversion and any gp_set_g). */
int gp_get_g(const gp_solver* s, double* g);

/* One FP64 pass over the field; synchronises; *out receives the observables. */
int gp_observables(gp_solver* s, gp_obs* out);

/* Integrated densities, Eq. 1 and its 3D analogues, FP64, synchronous.
 *   density1d: axis 0: out[i] = sum_{j,k} |psi|^2 dy dz   (out has nx entries)
 *              axis 1: out[j] = sum_{i,k} |psi|^2 dx dz   (ny entries)
 *              axis 2: out[k] = sum_{i,j} |psi|^2 dx dy   (nz entries)
 *   density2d: plane 0 (xy): out[j*nx+i] = sum_k |psi|^2 dz
 *              plane 1 (xz): out[k*nx+i] = sum_j |psi|^2 dy
 *              plane 2 (yz): out[k*ny+j] = sum_i |psi|^2 dx                        */
int gp_density1d(gp_solver* s, int axis, double* out);
int gp_density2d(gp_solver* s, int plane, double* out);

/* Wait for all queued work and report a status the kernels flagged since the last
 * check (GP_ERR_NONFINITE, GP_ERR_TIMEOUT), clearing it.                         */
int gp_sync(gp_solver* s);

/* Limit of the first bounded wait of a sweep kernel on each of its own shared-memory
 * copies (tile loads, row copies), in nanoseconds.  Default and maximum 2e9 (2 s);
 * first_wait_ns < 0 restores the default; 0 makes every first wait give up at once.  A wait that gives up sets the solver's timeout status, and
 * the kernel then waits (up to 2 s, whatever this limit) for the copies it still has
 * in flight before its blocks exit, so the device stays usable; the next gp_sync
 * returns GP_ERR_TIMEOUT and clears the status.  Meant for failure-detection tests:
 * a step whose waits gave up leaves the field partly updated.  Drops the solver's
 * step graphs (they hold the limit by value).  The paper has no counterpart: this
 * is failure detection of the GPU path.                                            */
int gp_set_wait_limit(gp_solver* s, long long first_wait_ns);

/* Per-sweep timing.  While enabled, every x / y / z sweep launch is bracketed by
 * CUDA events on the solver's stream.  gp_get_timing synchronises, adds the
 * elapsed milliseconds of the launches since the last read into ms[0..2] (x, y, z
 * sweep) and their counts into launches[0..2], then clears them.                 */
int gp_set_timing(gp_solver* s, int enable);
int gp_get_timing(gp_solver* s, double ms[3], long long launches[3]);

/* Layout facts of a solver in its current mode, for tests and tools:
 *   info[0] field pitch along x in elements, info[1] 1 if the field is complex,
 *   info[2..4] lines per shared-memory tile of the x / y / z tile kernels,
 *   info[5] device bytes in use,
 *   info[6] bit a set when sweep a (0 x, 1 y, 2 z) uses the FP32 kernels without
 *           shared-memory line tiles (decaying coupling cut below FP32 rounding, see
 *           gp_sweeps.cu), bit 3 + a when that kernel is the banded operator, bits
 *           8..11 the largest band half-width W, bits 12 + a when sweep a uses the
 *           FP64 line-streaming kernels (FP64 field; gp_sweeps64.cu), bit 15 when the
 *           banded x sweep holds each row in registers (k_sweep_x_reg),
 *   info[7] the truncation depth L of the streaming recurrences (0 when none).
 * GP_SWEEP_KERNELS=tile in the environment at gp_create time makes every sweep
 * use the tile kernels; =stream keeps the FP32 sweeps on the streaming recurrences
 * (=stream_x, =stream_yz: only x, only y and z).                                 */
int gp_get_info(const gp_solver* s, long long info[8]);

/* Observables of a field that sits in the caller's own device memory, computed
 * without allocating anything.  Meant for callers that cannot call cudaMalloc (which
 * gp_create needs): cudaMalloc synchronises the whole device and so stalls the other
 * streams of a latency-bound loop, it can fail while the free memory is held by
 * another allocator such as PyTorch's caching allocator, and some host programs that
 * load this library as a plugin do not allow device allocation in their callbacks.
 *   psi        device pointer; layout psi[k][j][i] with a row pitch of `pitch`
 *              elements (>= nx); prec GP_F64 (double) or GP_F32 (float); is_complex 1
 *              for interleaved (re, im) values.  The field is used as it is (no
 *              pending renormalisation).
 *   nx, ny, nz extents as in gp_params: 3..2048 each, or nz = 1 for a 2D field in
 *              the xy plane (then dz and lambda are ignored, z = 0, the cell area is
 *              dx dy and there is no z kinetic term, as for a 2D solver).
 *   dx..lambda, g   grid spacings, trap ratios and nonlinearity, as in gp_params.
 *   out        device pointer to 10 doubles, written in gp_obs order with the gp_obs
 *              definitions, once `stream` (a cudaStream_t, or NULL) reaches the work;
 *              the call itself returns as soon as the work is queued.
 * The reduction's scratch is a fixed 64 KiB array inside the library, held by every
 * GPU that loads the library until the process exits and shared by all calls: calls
 * whose work may overlap on the GPU (different streams with no ordering) race on it;
 * issue them on one stream.  The first call on a device looks up that array's device
 * address, which can load the library's GPU code: make this first call before any
 * stream capture begins.  Other extents or pitch < nx return GP_ERR_ARG,
 * with the reason in gp_last_error(NULL).  No cudaMalloc / cudaFree is called.
 * The paper has no counterpart; this is an operational variant of gp_observables.  */
int gp_observables_noalloc(const void* psi, int nx, int ny, int nz, long long pitch,
                           int prec, int is_complex, double dx, double dy, double dz,
                           double gamma, double nu, double lambda, double g, double* out,
                           void* stream);

/* Last error message of s, or, when s is NULL, of the calling thread's last failed
 * gp_create / gp_create_on / gp_workspace_bytes / gp_observables_noalloc.  Never NULL. */
const char* gp_last_error(const gp_solver* s);

/* Static text for a GP_* code. */
const char* gp_strerror(int code);

/* Physical units -> dimensionless nonlinearity (host only, no device).
 * g = 4 pi N a_s / l_osc with the s-wave scattering length given in Bohr radii
 * (a_0 = 5.29177210903e-11 m, CODATA 2018) and the oscillator length
 * l_osc = sqrt(hbar / (m omega_x)) in metres, the x-oscillator unit of length of the
 * equation's scaling.  natoms >= 0, a_s_bohr finite (negative: attractive),
 * l_osc_m > 0; GP_ERR_ARG otherwise.                                              */
int gp_units_g(double natoms, double a_s_bohr, double l_osc_m, double* g);

/* Oscillator length l_osc = sqrt(hbar / (m omega)) in metres of an atom of mass
 * mass_amu (unified atomic mass units, 1.66053906660e-27 kg) in a trap of angular
 * frequency omega (rad/s; 2 pi nu for a trap frequency nu in Hz).                 */
int gp_units_l_osc(double mass_amu, double omega, double* l_osc_m);

/* ---------------------------------------------------------------- pools
 * A pool keeps many FP32 solves of different grids resident in one device arena and
 * steps them together: batched uneven solves and the serving loop.  Every live slot
 * advances by the same SSCN step as a single FP32 solver (imaginary time on a real
 * field with renormalisation, or real time on a complex field), evaluated by one
 * batched launch per sweep direction and mode over packed work lists (rows of every
 * x line; blocks of every y / z line segment), the step captured as a CUDA graph.  A
 * slot's arithmetic depends only on its own parameters and the pool's launch shape,
 * not on which other slots are live.  All calls are synchronous unless stated.    */
typedef struct gp_pool gp_pool;

/* Arena bytes one solve with parameters p takes in a pool (host only). */
int gp_pool_slot_bytes(const gp_params* p, size_t* bytes);

/* Create a pool with an arena of arena_bytes (cudaMalloc'd on the current device) and
 * room for max_slots (1..4096) solves.  stream: a cudaStream_t the pool works on, or
 * NULL for a stream of its own (the legacy default stream cannot be captured).
 * GP_ERR_NOMEM when the arena cannot be allocated.                                */
int gp_pool_create(size_t arena_bytes, int max_slots, void* stream, gp_pool** out);
void gp_pool_destroy(gp_pool* pool);

/* Free arena bytes in total and in the largest free range. */
int gp_pool_free_bytes(const gp_pool* pool, size_t* free_bytes, size_t* largest);

/* Admit a solve: prec must be GP_F32, every extent >= 8, and dt / h^2 small enough
 * that the banded line operators need a half-width <= 8 (else GP_ERR_ARG).  The slot
 * starts from the g = 0 trap ground state exp(-(gamma x^2 + nu y^2 + lambda z^2)/2),
 * normalised, in imaginary time.  *slot receives its index.  GP_ERR_NOMEM when no
 * slot or no arena range of gp_pool_slot_bytes(p) is free.                          */
int gp_pool_add(gp_pool* pool, const gp_params* p, int* slot);

/* Retire a slot (after the work queued on the pool's stream) and free its range. */
int gp_pool_remove(gp_pool* pool, int slot);

/* Hand a slot over to real time: its field (with the pending renormalisation
 * applied) becomes complex; every later step is a real-time step.               */
int gp_pool_set_real_time(gp_pool* pool, int slot);

/* Replace a slot's nonlinearity g (quench). */
int gp_pool_set_g(gp_pool* pool, int slot, double g);

/* nsteps steps of every live slot in its own mode; GP_ERR_NONFINITE when a norm
 * became non-finite or zero.                                                      */
int gp_pool_step(gp_pool* pool, long nsteps);

/* Observables of one slot (gp_obs definitions as gp_observables). */
int gp_pool_observables(gp_pool* pool, int slot, gp_obs* out);

/* A slot's field to / from a caller-owned host FP64 buffer, layout
 * host[(k ny + j) nx + i] (interleaved re, im when complex).  set_psi also sets
 * the slot's mode (complex: real time).                                           */
int gp_pool_get_psi(gp_pool* pool, int slot, double* host, int as_complex);
int gp_pool_set_psi(gp_pool* pool, int slot, const double* host, int is_complex);

/* Launch shape: x_stages (2..8) rows in flight per warp of the x sweep, seg_turns
 * (1..8) turns of the 2W+1 ring per y / z segment.  gp_pool_tune times every pair
 * in {2,3,4} x {1,2,3,4} over steps_per_candidate steps on the live slots (their
 * state is saved before and restored after each candidate, so tuning advances no
 * solve), keeps the fastest and returns its time per step in *best_ms (NULL allowed).
 * gp_pool_set_graph(0) replaces the graph replay by direct launches.             */
int gp_pool_set_shape(gp_pool* pool, int x_stages, int seg_turns);
int gp_pool_tune(gp_pool* pool, int steps_per_candidate, double* best_ms);
int gp_pool_set_graph(gp_pool* pool, int enable);

/* info[0] live slots, [1] arena bytes in use, [2] x_stages, [3] seg_turns,
 * [4] bit 0: a step graph is instantiated, bit 1: the imaginary-time slots' x sweep
 * holds each row in registers (every such slot has rows of 16 m <= 512 points), bit 2:
 * the real-time slots' x sweep does (every such slot has rows of 8 m <= 256 complex
 * points), [5] launches per step, [6] free arena bytes, [7] largest free range.     */
int gp_pool_info(const gp_pool* pool, long long info[8]);
const char* gp_pool_last_error(const gp_pool* pool);

#ifdef __cplusplus
}
#endif
#endif

/*
 * gp_oracle.h -- plain FP64 CPU oracle for the split-step Crank-Nicolson (SSCN)
 * time step of the 3D Gross-Pitaevskii equation in an anisotropic harmonic trap.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code, header,
 * table or constant with the CUDA library; the two are checked against each other.
 *
 * Method (paper: program summary, "Solution method"; the imag3d / real3d program
 * summaries): the time-dependent GP equation is discretised in space and time and
 * propagated over small time steps by the split-step Crank-Nicolson scheme, in
 * imaginary time (real field, stationary state) or real time (complex field,
 * dynamics).  The paper prints neither the equation nor the discretisation; the
 * textbook forms written out in gp_oracle.c are the readings used here.
 *
 * Every function is single-threaded unless orc_set_threads(n > 1) was called, in
 * which case the independent line solves of one sweep run on n OpenMP threads.
 * Line solves never interact, so the result is bitwise the same for any n.
 */
#ifndef GP_ORACLE_H
#define GP_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Problem on an nx*ny*nz grid, layout psi[k][j][i] (x fastest), index
 * (k*ny + j)*nx + i.  Coordinates x_i = (i - (nx-1)/2) * hx (box centred on the
 * origin), same for y and z.  Homogeneous Dirichlet ghosts just outside the box.
 * Trap V = (gamma^2 x^2 + nu^2 y^2 + lambda^2 z^2) / 2.  nz = 1 is a 2D problem in
 * the xy plane: z = 0, no z solve, cell area hx hy in every sum.                 */
typedef struct {
  int nx, ny, nz;
  double hx, hy, hz;
  double dt;
  double gamma, nu, lambda;
  double g;
} orc_problem;

/* Number of OpenMP threads for line sweeps (1 = serial, the default).
 * Returns the count actually in effect (1 when built without OpenMP).      */
int orc_set_threads(int n);

/* g = 4 pi N a_s / l_osc  (a_s and l_osc in the same length unit). */
double orc_g_physical(double natoms, double a_s, double l_osc);

/* Grid coordinate (i - (n-1)/2) * h. */
double orc_coord(int i, int n, double h);

/* Thomas elimination coefficients for the CN system
 *   (1+2a) u_j - a (u_{j-1} + u_{j+1}) = d_j,  j = 0..n-1,  u_{-1} = u_n = 0,
 * with complex a = (are, aim).  cp[2n], m[2n] receive interleaved complex values. */
void orc_thomas_coeffs(int n, double are, double aim, double* cp, double* m);

/* One CN line update u = (I - a L)^-1 (I + a L) v, L = tridiag(1,-2,1) with zero
 * ghosts, in place on the interleaved complex line v[2n].                        */
void orc_cn_line(int n, double are, double aim, double* v);

/* Normalised Gaussian exp(-(wx x^2 + wy y^2 + wz z^2)/2), normalised on the grid
 * (sum |psi|^2 dV = 1).  psi: real field of nx*ny*nz doubles.                    */
void orc_init_gaussian(const orc_problem* p, double wx, double wy, double wz, double* psi);

/* nsteps imaginary-time SSCN steps on a real field, renormalising after each.
 * Returns 0, or -4 when the norm became non-finite or zero.                      */
int orc_step_imag(const orc_problem* p, double* psi, long nsteps);

/* nsteps real-time SSCN steps on a complex field psi[2*N] (interleaved re, im). */
int orc_step_real(const orc_problem* p, double* psi, long nsteps);

/* Strang-split variants: half pointwise substep, the three CN solves, half
 * pointwise substep (then the renormalisation in imaginary time).                */
int orc_step_imag_strang(const orc_problem* p, double* psi, long nsteps);
int orc_step_real_strang(const orc_problem* p, double* psi, long nsteps);

/* Observables of psi (real: N doubles; complex: 2N interleaved).
 * out[10] = norm, mu, energy, ekin, epot, eint, rms_x, rms_y, rms_z, rms_r.       */
void orc_observables(const orc_problem* p, const double* psi, int is_complex, double* out);

/* Integrated densities (Eq. 1 and its 3D analogues).
 * density1d: axis 0/1/2 -> out[nx] / out[ny] / out[nz].
 * density2d: plane 0 (xy) out[j*nx+i], 1 (xz) out[k*nx+i], 2 (yz) out[k*ny+j].   */
void orc_density1d(const orc_problem* p, const double* psi, int is_complex, int axis, double* out);
void orc_density2d(const orc_problem* p, const double* psi, int is_complex, int plane, double* out);

#ifdef __cplusplus
}
#endif
#endif

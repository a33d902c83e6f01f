/*
 * FP64 CPU oracle for the D3Q19-MRT lattice Boltzmann permeability solver of
 * Rao & Schaefer, "Lattice Boltzmann Models for Micro-tomographic
 * Pore-spaces" (arXiv:1902.11193).
 *
 * TEST INFRASTRUCTURE ONLY.  This is the plain, slow reference that the CUDA
 * path is checked against.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline arm may load it; the product library never does.
 * It shares no code, header, table or helper with the CUDA path.
 *
 * Conventions (the paper prints none of these; the readings are listed in the
 * design notes):
 *   velocities  i = 0 rest; 1..6 = +x,-x,+y,-y,+z,-z; 7..18 = (1,1,0),
 *               (-1,-1,0),(1,-1,0),(-1,1,0),(1,0,1),(-1,0,-1),(1,0,-1),
 *               (-1,0,1),(0,1,1),(0,-1,-1),(0,1,-1),(0,-1,1)
 *   node index  n = x + Lx*(y + Ly*z); mask 1 = solid, 0 = fluid
 *   populations f[i*N + n], unshifted (rest state f_i = w_i, rho0 = 1)
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORA_SET_A = 0, ORA_SET_B, ORA_SET_C, ORA_SET_D, ORA_SET_E, ORA_SET_SRT };

/* Lattice constants: c[19][3], w[19], opposite[19]. */
void ora_lattice(int32_t c[19 * 3], double w[19], int32_t opp[19]);
/* Dense moment matrix M[19][19] (row k = moment k, Sec. 2.2.1 order). */
void ora_moment_matrix(double M[19 * 19]);
/* Relaxation rates s[19] of Table 2 for (set, tau, Lambda). Returns 0 or -1. */
int ora_rates(int set, double tau, double Lambda, double s[19]);
/* Equilibrium moments, eq. (MRT Equi), for density rho and shifted momentum j. */
void ora_meq(double rho, const double j[3], int linear, double meq[19]);
/* Guo forcing populations, eq. (Guo_Forcing), for velocity u and force F. */
void ora_guo_populations(const double u[3], const double F[3], int linear, double Fi[19]);
/* Forcing moments m^F = M . F_i (the literal matrix-vector product). */
void ora_force_moments(const double u[3], const double F[3], int linear, double mF[19]);
/* One MRT collision of a single node: f -> f*, eq. (MRT-LBE). */
void ora_collide(const double f[19], const double s[19], const double F[3], int linear,
                 double fout[19]);

/* Two-relaxation-time collision in link form with the even rate s_plus and
 * the odd rate s_minus (the MRT collision for rates with one even and one odd
 * value: Sets B, E and SRT). */
void ora_trt_collide(const double f[19], double s_plus, double s_minus, const double F[3],
                     int linear, double fout[19]);
/* Link table of a mask: fluid list, pull neighbours (x - c_i) and bounceback
 * bits.  fluid_idx[Nf], nbr[18][Nf] (entry for direction i at (i-1)*Nf + n,
 * -1 where x - c_i is solid), bbmask[Nf] (bit i set iff x - c_i is solid),
 * links[19] (per-direction count of bounceback links).  Any output may be
 * NULL.  Returns Nf. */
int64_t ora_links(const uint8_t *mask, const int32_t dims[3], int32_t *fluid_idx,
                  int32_t *nbr, uint32_t *bbmask, int64_t links[19]);

typedef struct ora_solver ora_solver;
ora_solver *ora_create(const uint8_t *mask, const int32_t dims[3], const double s[19],
                       const double F[3], int linear);
void ora_destroy(ora_solver *h);
/* n pull-stream + collide steps.  If U is non-NULL it receives the mean
 * velocity of the streamed state collided in the last step. */
void ora_step(ora_solver *h, int64_t n, double U[3]);
/* Mean velocity (over all N voxels, solids count as 0) of the current state
 * after streaming, without advancing: U = (1/N) sum_fluid (sum_i c_i f_i + F/2). */
void ora_mean_velocity(ora_solver *h, double U[3]);
/* Velocity field u[3][N] of the streamed current state (0 in solids). */
void ora_velocity(ora_solver *h, double *u);
void ora_get_f(ora_solver *h, double *f);
void ora_set_f(ora_solver *h, const double *f);
int64_t ora_steps_done(ora_solver *h);
/* Steps in chunks of K until |U_b - U_a| <= tol |U_b| for the mean x-velocity
 * of the last two steps of a chunk, or max_steps.  Returns 0 converged, 1 not
 * converged, 2 non-finite. */
int ora_run_to_convergence(ora_solver *h, double tol, int64_t K, int64_t max_steps,
                           int64_t *steps, double U[3]);
/* The same with a choice of stopping rule: rule 0 is the rule above; rule 1
 * applies it to the mean over two consecutive steps, measured in the last
 * three steps of a chunk (K >= 3): Ubar_b = (U_b + U_c)/2 against
 * Ubar_a = (U_a + U_b)/2.  U receives the measure the rule stopped on. */
int ora_run_to_convergence_rule(ora_solver *h, double tol, int64_t K, int64_t max_steps,
                                int rule, int64_t *steps, double U[3]);
/* Voxel flags of the image analysis (Sec. 3): flags[N] = 0 fluid, 1 solid
 * voxel with a fluid voxel among its 18 link neighbours (bounceback voxel),
 * 2 other solid.  Returns the number of bounceback voxels. */
int64_t ora_flags(const uint8_t *mask, const int32_t dims[3], uint8_t *flags);
/* Bounceback scheme: 0 halfway (default: the wall at the half-link, applied
 * in the pull), 1 full-way (Sec. 3: bounceback voxels receive the populations
 * streamed into them and return each along the opposite link in the next
 * step, without collision or force; fluid voxels stream from every
 * neighbour).  The adjoint and the field-streaming functions assume halfway
 * bounceback.  Returns 0, or -1 for a bad mode. */
int ora_set_bounceback(ora_solver *h, int mode);
/* Bounded domain (Sec. 2.4): pressure_x = 1 makes the x faces Zou-He
 * density boundaries (inlet x = 0 at rho_in, outlet x = Lx-1 at rho_out;
 * requires F = 0 and Lx >= 2); symmetry bit 0 / bit 1 makes the y / z faces
 * symmetry (mirror) planes half a link outside the outer nodes.  Unset keeps
 * a direction periodic.  Halfway bounceback only; the adjoint and the
 * field-streaming functions assume the periodic domain.  Returns 0 or -1. */
int ora_set_domain(ora_solver *h, int pressure_x, double rho_in, double rho_out,
                   int symmetry);
void ora_set_threads(int n);
int ora_get_threads(void);

/* Rates of the TRT-like sets (B, D, E) with the odd rates given by their
 * magic parameters: s_q from Lambda_q, s_m from Lambda_m (eq. Magic param),
 * even rates s_nu = 1/tau.  Set B is (3/16, 3/16), Set D (3/16, 3/8), Set E
 * (Lambda, Lambda). */
int ora_rates_magic(double tau, double Lq, double Lm, double s[19]);

/* Streaming as a linear map on whole fields [19][N]: out = S in (pull with
 * halfway bounceback) and out = S^T in (its transpose, S^-1).  Solid nodes
 * are copied through. */
void ora_stream_field(ora_solver *h, const double *in, double *out);
void ora_unstream_field(ora_solver *h, const double *in, double *out);
/* One adjoint step without source: out = J_C(h)^T S^T in, where h = S f* is
 * the streamed current state and J_C the per-node collision Jacobian. */
void ora_adjoint_apply(ora_solver *h, const double *in, double *out);

/* Steady fixed-point adjoint of k along the drive (largest |F_j|):
 * psi = J_C^T S^T psi + dk/dh, iterated from psi = dk/dh until the largest
 * change over two iterations is <= tol times the largest |psi| (checked every
 * K iterations).  The linearisation point h is the mean of the streamed
 * states of the current and the next step (the solver advances one step),
 * and the gradient uses the mean of the last two iterates: both means remove
 * the period-2 component that bounceback in thin gaps can leave in either
 * iteration.
 * The gradient is dk/dtheta = dJ/dtheta + (S^T psi) . dC/dtheta.
 * (set, tau, Lambda) must be the parameters the solver's rates came from.
 * grad = {dk/dtau, dk/dLambda, dk/dLambda_q, dk/dLambda_m, dk/dF_x,
 * dk/dF_y, dk/dF_z}; the Lambda entries are NaN for sets without magic
 * parameters (A, C, SRT).  Returns 0, 1 (not converged) or -1. */
int ora_adjoint(ora_solver *h, int set, double tau, double Lambda, double tol, int64_t K,
                int64_t max_iter, double grad[7], int64_t *iters);
/* Gradient of the permeability after n more steps (the solver advances n
 * steps): reverse accumulation through every step, all states kept.  grad as
 * for ora_adjoint.  Returns 0, or -1 for bad input. */
int ora_adjoint_transient(ora_solver *h, int set, double tau, double Lambda, int64_t n,
                          double grad[7]);

#ifdef __cplusplus
}
#endif
#endif

/*
 * lbm_oracle.h -- FP64 CPU oracle of the coupled lattice Boltzmann /
 * rigid-body swimmer step (Pickl et al., "All good things come in threes",
 * arXiv:1108.0786, Sections 2.1-2.3 and 3.1-3.3, Algorithms 1 and 2).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the plain, slow reference that
 * the GPU library is checked against.  Only the test-suite, the smoke check
 * and the CPU-baseline leg of the benchmark may load it.  It shares no code,
 * header, table or helper with the GPU library.
 *
 * Conventions (lattice units, dx = dt = 1, rest density 1):
 *   - cell (x, y, z) has its centre at the integer point (x, y, z) and linear
 *     index c = (z * ny + y) * nx + x;
 *   - populations are stored as [19][cells] in the velocity order
 *       0:( 0, 0, 0)
 *       1:(+1, 0, 0)  2:(-1, 0, 0)  3:( 0,+1, 0)  4:( 0,-1, 0)
 *       5:( 0, 0,+1)  6:( 0, 0,-1)
 *       7:(+1,+1, 0)  8:(-1,-1, 0)  9:(+1,-1, 0) 10:(-1,+1, 0)
 *      11:(+1, 0,+1) 12:(-1, 0,-1) 13:(+1, 0,-1) 14:(-1, 0,+1)
 *      15:( 0,+1,+1) 16:( 0,-1,-1) 17:( 0,+1,-1) 18:( 0,-1,+1)
 *   - a body state is 13 doubles: position[3], unit quaternion (w,x,y,z)[4],
 *     velocity[3], angular velocity[3]; the body-frame x axis is the capsule
 *     axis and the drive axis.
 *
 * Every call returns 0 or a negative REF_E_* code.
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define REF_OK            0
#define REF_E_ARG        -1
#define REF_E_OOM        -2
#define REF_E_OVERLAP    -3
#define REF_E_OUTSIDE    -4
#define REF_E_NAN        -5
#define REF_E_STATE      -9

#define REF_BC_PERIODIC_X 1
#define REF_BC_PERIODIC_Y 2
#define REF_BC_PERIODIC_Z 4

#define REF_SHAPE_SPHERE  0
#define REF_SHAPE_CAPSULE 1

#define REF_OPT_NO_FLUID  1   /* bodies only: no mapping, no hydrodynamic force */
#define REF_OPT_AVERAGE_FORCE 2  /* rigid-body step with the mean load of steps n and n-1 */

#define REF_FIELD_RHO   0     /* double[cells] */
#define REF_FIELD_U     1     /* double[3][cells] */
#define REF_FIELD_FLAGS 2     /* unsigned char[cells]: 0 fluid, 1 + body id if solid */
#define REF_FIELD_POP   3     /* double[19][cells]: post-collision populations */

typedef struct ref_lbm ref_lbm;

int  lbm_ref_create(int nx, int ny, int nz, double tau, int bc, ref_lbm **out);
int  lbm_ref_create_ex(int nx, int ny, int nz, double tau, int bc,
                       const double g[3], int options, ref_lbm **out);
int  lbm_ref_destroy(ref_lbm *h);
int  lbm_ref_add_body(ref_lbm *h, int shape, double radius, double length,
                      double mass, const double pos[3], const double orient[4]);
int  lbm_ref_add_spring(ref_lbm *h, int i, int j, double k, double rest,
                        double damping);
int  lbm_ref_set_drive(ref_lbm *h, int body, double amp, double freq,
                       double phase);
int  lbm_ref_set_drive_window(ref_lbm *h, int term, double t_off);
/* direction of a drive term as a body-frame vector (default 1, 0, 0: the
 * body x axis), used unnormalised; before the first step */
int  lbm_ref_set_drive_axis(ref_lbm *h, int term, const double axis[3]);
int  lbm_ref_set_body_state(ref_lbm *h, int body, const double state[13]);
int  lbm_ref_step(ref_lbm *h, int n);
/* running time average of the velocity field from the next step on, and
 * its mean [3][cells] with the number of steps averaged */
int  lbm_ref_average_begin(ref_lbm *h);
int  lbm_ref_average_get(ref_lbm *h, double *out, long *steps);
int  lbm_ref_get_bodies(ref_lbm *h, double *out);
int  lbm_ref_get_forces(ref_lbm *h, double *out);
int  lbm_ref_get_fields(ref_lbm *h, int what, void *out);
int  lbm_ref_set_pop(ref_lbm *h, const double *pop);
long lbm_ref_steps_done(ref_lbm *h);
int  lbm_ref_lattice(int *e /* [19][3] */, double *w /* [19] */);
int  lbm_ref_equilibrium(double rho, const double u[3], double *out /* [19] */);
int  lbm_ref_body_props(ref_lbm *h, int b, double *out /* volume, I1, I2, I3 */);
int  lbm_ref_num_threads(void);
int  lbm_ref_set_num_threads(int n);
/* Reverse mode: advances n steps (recording every one), then returns the
 * gradient of J = sum_b seed[b] . state_b(after the n steps) (seed: nb x 13)
 * with respect to the body states at the start (grad_state, nb x 13) and the
 * state before it (grad_prev: the wall velocities of the first stream; zero
 * and folded into grad_state when the run starts at the first step), the
 * populations entering the first step (grad_pop, 19 x cells), the drive
 * terms (grad_drive, nd x 2: amp, phase), the springs (grad_spring, ns x 3:
 * k, rest, damping) and the bodies (grad_body, nb x 5: mass, the three
 * principal moments of inertia, volume), with the obstacle maps of the run
 * held fixed.  Any output may be NULL. */
int  lbm_ref_adjoint(ref_lbm *h, int n, const double *seed, double *grad_state,
                     double *grad_prev, double *grad_pop, double *grad_drive,
                     double *grad_spring, double *grad_body);
/* running digest of the obstacle map of every step taken so far */
unsigned long long lbm_ref_flag_digest(ref_lbm *h);
const char *lbm_ref_last_error(ref_lbm *h);

#ifdef __cplusplus
}
#endif
#endif

/*
 * lbm_oracle.c -- FP64 CPU oracle of one coupled D3Q19 lattice Boltzmann /
 * rigid-body time step with moving obstacles, written from Pickl et al.,
 * "All good things come in threes -- Three beads learn to swim with lattice
 * Boltzmann and a rigid body solver" (arXiv:1108.0786).
 *
 * TEST INFRASTRUCTURE ONLY: this is the plain, slow, obviously-correct
 * reference that the GPU library is checked against.  Only tests, the smoke
 * check and the CPU-baseline leg of the benchmark may load it.  It shares no
 * code, header, table or constant generator with the GPU library.
 *
 * One call of lbm_ref_step advances the state by the coupled step of
 * Algorithm 2, in the paper's order:
 *   1. map every body onto the lattice (Sec. 2.3, "cell centre inside an
 *      object"), turning fluid cells into obstacle cells and reconstructing
 *      the populations of uncovered cells from f_eq(rho_avg, u_w);
 *   2. stream (Eq. 3) with velocity-corrected bounce-back at obstacle links
 *      (moving-wall rule of Sec. 2.3; Eq. 4 for the static channel walls) and
 *      collide (LBGK, Eq. 1-2);
 *   3. momentum-exchange force on each body (Eq. hydroF) and its torque;
 *   4. the driving forces of the cycling strategy (Eq. FB1-FB3);
 *   5. the rigid-body time step (Algorithm 1) with the damped springs
 *      (Eq. osci_i, osci_j) and the total force (Eq. totalFSwimmer).
 *
 * Readings taken where the paper is silent or garbled (each one is listed in
 * the design notes of the repository):
 *   - f_eq is the standard second-order D3Q19 equilibrium with weights
 *     1/3, 1/18, 1/36 (the paper cites Qian et al. but prints no formula);
 *   - rho_w in the moving-wall rule is the density sum_a f~_a(x_f) of the
 *     fluid cell of the link;
 *   - the sum "alpha = 1..19" of Eq. hydroF runs over the 18 moving
 *     directions of the links (x_f, alpha) whose end x_f + e_alpha is solid;
 *   - torque is taken about the body centre with the link force applied at
 *     the link midpoint x_f + e_alpha / 2 (the paper gives no torque);
 *   - a cell is solid iff its centre satisfies |d|^2 <= r^2 (sphere) or
 *     |d - s a|^2 <= r^2 with s the clamped axial coordinate (capsule), d
 *     the periodic minimum-image offset from the body centre;
 *   - the stream into step n uses the obstacle flags and the body state of
 *     step n-1; the force of step n uses flags and state of step n, so the
 *     force is exactly the momentum the next stream exchanges;
 *   - an uncovered cell takes f_eq(rho_avg, u_w(x)) for all 19 directions,
 *     rho_avg being the mean density of the D3Q19 neighbours that are fluid
 *     in both the previous and the current flag epoch (1 if none);
 *   - cells that become solid drop their populations;
 *   - bodies advance by semi-implicit Euler with dt = 1: V += F/m, X += V,
 *     Omega += I_world^-1 T, q += (0,Omega) q / 2 then renormalised;
 *   - drive term: F = amp sin(2 pi freq t - phase) along a body-frame axis
 *     (default the body x axis) for phase/(2 pi freq) <= t < t_off, zero
 *     otherwise (the paper delays the third body by T/4, Sec. 3.3 and 5.1);
 *   - body force g (a force density) enters the fluid through Guo's forcing
 *     term and the bodies as g times their volume;
 *   - option REF_OPT_AVERAGE_FORCE (not in the paper): the rigid-body step
 *     takes the mean hydrodynamic force and torque of steps n and n-1, a
 *     stabiliser of the explicit coupling for bodies near or below the
 *     fluid's density.
 *
 * Collision, stream and field exports are parallel over cells with OpenMP
 * when compiled with -fopenmp; every loop that sums in a particular order
 * (the density average of a refill, the force and torque sums) is serial, so
 * results do not depend on the thread count.  The force of a body sums its
 * links in z, y, x order over the body's bounding box, then by direction.
 */
#include "lbm_oracle.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 19
#define MAX_BODIES 254

/* D3Q19 velocity set (Sec. 2.1, Qian et al.) in the order documented in the
 * header, and the standard weights: 1/3 rest, 1/18 axis, 1/36 diagonal. */
static const int EX[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
static const int EY[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
static const int EZ[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
static const double W[Q] = {
    1.0 / 3.0,
    1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

/* index of the opposite direction, e_opp(a) = -e_a, filled at creation */
static int OPP[Q];

static void fill_opposite(void)
{
    for (int a = 0; a < Q; ++a)
        for (int b = 0; b < Q; ++b)
            if (EX[b] == -EX[a] && EY[b] == -EY[a] && EZ[b] == -EZ[a]) OPP[a] = b;
}

typedef struct {
    int shape;
    double r, l, m;
    double inertia[3];   /* principal moments in the body frame */
    double volume;
    double X[3], q[4], V[3], Om[3];
} body_t;

typedef struct { int i, j; double k, rest, gamma; } spring_t;
typedef struct { int body; double amp, freq, phase, t_off, axis[3]; } drive_t;

struct ref_lbm {
    int nx, ny, nz, bc, options;
    long C;
    double tau, g[3];
    double *F;              /* pre-collision populations f     [Q][C] */
    double *G;              /* post-collision populations f~   [Q][C] */
    short *bid_now, *bid_prev;  /* body id of solid cells, -1 for fluid */
    int nb, ns, nd;
    body_t body[MAX_BODIES];
    body_t body_prev[MAX_BODIES];   /* body state of the previous step */
    spring_t *spring;
    drive_t *drive;
    double Fh[MAX_BODIES][3], Th[MAX_BODIES][3];
    double Fh_prev[MAX_BODIES][3], Th_prev[MAX_BODIES][3];   /* load of the previous step */
    long step;
    int started;
    unsigned long long flag_digest;   /* running digest of every step's obstacle map */
    struct tape *tape;                /* recording for the reverse sweep, or NULL */
    double *avg_sum;                  /* running sum of the velocity [3][C], or NULL */
    long avg_steps;                   /* steps added to it */
    int avg_on;
    char err[256];
};

static int fail(ref_lbm *h, int code, const char *msg)
{
    if (h) snprintf(h->err, sizeof h->err, "%s", msg);
    return code;
}

static long cell(const ref_lbm *h, int x, int y, int z)
{
    return ((long)z * h->ny + y) * h->nx + x;
}

/* Wrap coordinate i on an axis of n cells: periodic axes wrap, walled axes
 * report -1 for a coordinate outside the domain. */
static int wrap(int i, int n, int periodic)
{
    if (i >= 0 && i < n) return i;
    if (!periodic) return -1;
    i %= n;
    return i < 0 ? i + n : i;
}

static double min_image(double d, int n, int periodic)
{
    if (periodic) d -= n * rint(d / n);
    return d;
}

/* ---- small vector / rotation helpers ---------------------------------- */

static void rot_matrix(const double q[4], double R[3][3])
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z);     R[0][2] = 2 * (x * z + w * y);
    R[1][0] = 2 * (x * y + w * z);     R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
    R[2][0] = 2 * (x * z - w * y);     R[2][1] = 2 * (y * z + w * x);     R[2][2] = 1 - 2 * (x * x + y * y);
}

static void cross(const double a[3], const double b[3], double c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* offset of lattice point p from the body centre, periodic minimum image */
static void body_offset(const ref_lbm *h, const body_t *b, const double p[3], double d[3])
{
    d[0] = min_image(p[0] - b->X[0], h->nx, h->bc & REF_BC_PERIODIC_X);
    d[1] = min_image(p[1] - b->X[1], h->ny, h->bc & REF_BC_PERIODIC_Y);
    d[2] = min_image(p[2] - b->X[2], h->nz, h->bc & REF_BC_PERIODIC_Z);
}

/* "cell centre inside the object" (Sec. 2.3), closed test on the surface */
static int inside(const ref_lbm *h, const body_t *b, int x, int y, int z)
{
    double p[3] = {x, y, z}, d[3];
    body_offset(h, b, p, d);
    if (b->shape == REF_SHAPE_SPHERE)
        return d[0] * d[0] + d[1] * d[1] + d[2] * d[2] <= b->r * b->r;
    /* capsule: cylinder of length l along the body x axis plus two
     * hemispherical caps; distance to the axis segment <= r */
    double R[3][3];
    rot_matrix(b->q, R);
    double a[3] = {R[0][0], R[1][0], R[2][0]};
    double s = d[0] * a[0] + d[1] * a[1] + d[2] * a[2];
    if (s > 0.5 * b->l) s = 0.5 * b->l;
    if (s < -0.5 * b->l) s = -0.5 * b->l;
    double e0 = d[0] - s * a[0], e1 = d[1] - s * a[1], e2 = d[2] - s * a[2];
    return e0 * e0 + e1 * e1 + e2 * e2 <= b->r * b->r;
}

/* velocity of the object at lattice point p: u_w = V + Omega x (p - X) */
static void wall_velocity(const ref_lbm *h, const body_t *b, const double p[3], double u[3])
{
    double d[3], c[3];
    body_offset(h, b, p, d);
    cross(b->Om, d, c);
    u[0] = b->V[0] + c[0];
    u[1] = b->V[1] + c[1];
    u[2] = b->V[2] + c[2];
}

/* standard second-order equilibrium of direction a */
static double feq(int a, double rho, const double u[3])
{
    double eu = EX[a] * u[0] + EY[a] * u[1] + EZ[a] * u[2];
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return W[a] * rho * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
}

/* velocity of cell c from the post-collision populations G:
 * u = (sum_a e_a f~_a - g/2) / rho, the velocity Guo's collision used;
 * 0 in obstacle cells.  Returns rho (1 in obstacle cells). */
static double cell_velocity(const ref_lbm *h, long c, int solid, double u[3])
{
    double rho = 0.0, m[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < Q; ++a) {
        double f = h->G[a * h->C + c];
        rho += f;
        m[0] += EX[a] * f; m[1] += EY[a] * f; m[2] += EZ[a] * f;
    }
    for (int i = 0; i < 3; ++i) u[i] = solid ? 0.0 : (m[i] - 0.5 * h->g[i]) / rho;
    return solid ? 1.0 : rho;
}

/* ---- creation ------------------------------------------------------------ */

int lbm_ref_create_ex(int nx, int ny, int nz, double tau, int bc,
                      const double g[3], int options, ref_lbm **out)
{
    if (!out) return REF_E_ARG;
    *out = NULL;
    fill_opposite();
    if (nx < 1 || ny < 1 || nz < 1 || !(tau > 0.5) || bc < 0 || bc > 7 ||
        (options & ~(REF_OPT_NO_FLUID | REF_OPT_AVERAGE_FORCE)))
        return REF_E_ARG;
    ref_lbm *h = calloc(1, sizeof *h);
    if (!h) return REF_E_OOM;
    h->nx = nx; h->ny = ny; h->nz = nz; h->bc = bc; h->tau = tau;
    h->options = options;
    h->C = (long)nx * ny * nz;
    if (g) { h->g[0] = g[0]; h->g[1] = g[1]; h->g[2] = g[2]; }
    h->F = malloc(sizeof(double) * Q * h->C);
    h->G = malloc(sizeof(double) * Q * h->C);
    h->bid_now = malloc(sizeof(short) * h->C);
    h->bid_prev = malloc(sizeof(short) * h->C);
    if (!h->F || !h->G || !h->bid_now || !h->bid_prev) {
        lbm_ref_destroy(h);
        return REF_E_OOM;
    }
    /* fluid at rest: f = f_eq(1, 0) = w_a everywhere; no obstacles yet */
    for (int a = 0; a < Q; ++a)
        for (long c = 0; c < h->C; ++c) h->F[a * h->C + c] = h->G[a * h->C + c] = W[a];
    for (long c = 0; c < h->C; ++c) h->bid_now[c] = h->bid_prev[c] = -1;
    *out = h;
    return REF_OK;
}

int lbm_ref_create(int nx, int ny, int nz, double tau, int bc, ref_lbm **out)
{
    return lbm_ref_create_ex(nx, ny, nz, tau, bc, NULL, 0, out);
}

int lbm_ref_destroy(ref_lbm *h)
{
    if (!h) return REF_OK;
    free(h->F); free(h->G); free(h->bid_now); free(h->bid_prev);
    free(h->spring); free(h->drive); free(h->avg_sum);
    free(h);
    return REF_OK;
}

int lbm_ref_add_body(ref_lbm *h, int shape, double radius, double length,
                     double mass, const double pos[3], const double orient[4])
{
    if (!h || !pos) return REF_E_ARG;
    if (h->started) return fail(h, REF_E_STATE, "bodies must be added before the first step");
    if (h->nb >= MAX_BODIES) return fail(h, REF_E_ARG, "too many bodies");
    if (shape != REF_SHAPE_SPHERE && shape != REF_SHAPE_CAPSULE)
        return fail(h, REF_E_ARG, "unknown shape");
    if (!(radius > 0) || !(mass > 0) || length < 0 || (shape == REF_SHAPE_SPHERE && length != 0))
        return fail(h, REF_E_ARG, "bad body dimensions");
    body_t *b = &h->body[h->nb];
    memset(b, 0, sizeof *b);
    b->shape = shape; b->r = radius; b->l = length; b->m = mass;
    for (int i = 0; i < 3; ++i) b->X[i] = pos[i];
    if (orient) {
        double n = sqrt(orient[0] * orient[0] + orient[1] * orient[1] +
                        orient[2] * orient[2] + orient[3] * orient[3]);
        if (!(n > 0)) return fail(h, REF_E_ARG, "zero quaternion");
        for (int i = 0; i < 4; ++i) b->q[i] = orient[i] / n;
    } else {
        b->q[0] = 1.0;
    }
    double r = radius, l = length;
    if (shape == REF_SHAPE_SPHERE) {
        b->volume = 4.0 / 3.0 * M_PI * r * r * r;
        b->inertia[0] = b->inertia[1] = b->inertia[2] = 0.4 * mass * r * r;
    } else {
        /* uniform solid capsule: cylinder (length l) + two hemispheres */
        double vc = M_PI * r * r * l, vh = 2.0 / 3.0 * M_PI * r * r * r;
        b->volume = vc + 2.0 * vh;
        double mc = mass * vc / b->volume, mh = mass * vh / b->volume;
        b->inertia[0] = 0.5 * mc * r * r + 2.0 * (0.4 * mh * r * r);
        b->inertia[1] = b->inertia[2] =
            mc * (r * r / 4.0 + l * l / 12.0) +
            2.0 * mh * (0.4 * r * r + l * l / 4.0 + 3.0 * l * r / 8.0);
    }
    return h->nb++;
}

int lbm_ref_add_spring(ref_lbm *h, int i, int j, double k, double rest, double damping)
{
    if (!h) return REF_E_ARG;
    if (h->started) return fail(h, REF_E_STATE, "springs must be added before the first step");
    if (i < 0 || j < 0 || i >= h->nb || j >= h->nb || i == j || k < 0 || rest < 0 || damping < 0)
        return fail(h, REF_E_ARG, "bad spring");
    spring_t *s = realloc(h->spring, sizeof *s * (h->ns + 1));
    if (!s) return REF_E_OOM;
    h->spring = s;
    s[h->ns] = (spring_t){i, j, k, rest, damping};
    return h->ns++;
}

int lbm_ref_set_drive(ref_lbm *h, int body, double amp, double freq, double phase)
{
    if (!h) return REF_E_ARG;
    if (h->started) return fail(h, REF_E_STATE, "drives must be added before the first step");
    if (body < 0 || body >= h->nb || !(freq > 0) || phase < 0)
        return fail(h, REF_E_ARG, "bad drive");
    drive_t *d = realloc(h->drive, sizeof *d * (h->nd + 1));
    if (!d) return REF_E_OOM;
    h->drive = d;
    d[h->nd] = (drive_t){body, amp, freq, phase, INFINITY, {1.0, 0.0, 0.0}};
    return h->nd++;
}

int lbm_ref_set_drive_axis(ref_lbm *h, int term, const double axis[3])
{
    if (!h || !axis || term < 0 || term >= h->nd) return REF_E_ARG;
    if (h->started) return fail(h, REF_E_STATE, "drive axes must be set before the first step");
    for (int i = 0; i < 3; ++i) h->drive[term].axis[i] = axis[i];
    return REF_OK;
}

int lbm_ref_set_drive_window(ref_lbm *h, int term, double t_off)
{
    if (!h || term < 0 || term >= h->nd) return REF_E_ARG;
    h->drive[term].t_off = t_off;
    return REF_OK;
}

int lbm_ref_set_body_state(ref_lbm *h, int b, const double s[13])
{
    if (!h || !s || b < 0 || b >= h->nb) return REF_E_ARG;
    body_t *B = &h->body[b];
    double n = sqrt(s[3] * s[3] + s[4] * s[4] + s[5] * s[5] + s[6] * s[6]);
    if (!(n > 0)) return fail(h, REF_E_ARG, "zero quaternion");
    for (int i = 0; i < 3; ++i) { B->X[i] = s[i]; B->V[i] = s[7 + i]; B->Om[i] = s[10 + i]; }
    for (int i = 0; i < 4; ++i) B->q[i] = s[3 + i] / n;
    return REF_OK;
}

int lbm_ref_set_pop(ref_lbm *h, const double *pop)
{
    if (!h || !pop) return REF_E_ARG;
    memcpy(h->G, pop, sizeof(double) * Q * h->C);
    return REF_OK;
}

/* ---- step 1: map the bodies onto the lattice (Sec. 2.3) ------------------ */

static int body_outside_walls(const ref_lbm *h, const body_t *b)
{
    double R[3][3];
    rot_matrix(b->q, R);
    int n[3] = {h->nx, h->ny, h->nz};
    int per[3] = {h->bc & REF_BC_PERIODIC_X, h->bc & REF_BC_PERIODIC_Y, h->bc & REF_BC_PERIODIC_Z};
    for (int k = 0; k < 3; ++k) {
        if (per[k]) continue;
        double ext = b->r + (b->shape == REF_SHAPE_CAPSULE ? 0.5 * b->l * fabs(R[k][0]) : 0.0);
        /* the walls sit half a cell outside the first and last cell centres */
        if (b->X[k] - ext < -0.5 || b->X[k] + ext > n[k] - 0.5) return 1;
    }
    return 0;
}

static int map_bodies(ref_lbm *h, short *bid)
{
    for (long c = 0; c < h->C; ++c) bid[c] = -1;
    if (h->options & REF_OPT_NO_FLUID) return REF_OK;
    int per[3] = {h->bc & REF_BC_PERIODIC_X, h->bc & REF_BC_PERIODIC_Y, h->bc & REF_BC_PERIODIC_Z};
    for (int k = 0; k < h->nb; ++k) {
        const body_t *b = &h->body[k];
        if (body_outside_walls(h, b))
            return fail(h, REF_E_OUTSIDE, "a body crosses a wall of the domain");
        double ext = b->r + 0.5 * b->l;   /* bounding-sphere radius */
        for (int iz = (int)floor(b->X[2] - ext) - 1; iz <= (int)ceil(b->X[2] + ext) + 1; ++iz) {
            int z = wrap(iz, h->nz, per[2]);
            if (z < 0) continue;
            for (int iy = (int)floor(b->X[1] - ext) - 1; iy <= (int)ceil(b->X[1] + ext) + 1; ++iy) {
                int y = wrap(iy, h->ny, per[1]);
                if (y < 0) continue;
                for (int ix = (int)floor(b->X[0] - ext) - 1; ix <= (int)ceil(b->X[0] + ext) + 1; ++ix) {
                    int x = wrap(ix, h->nx, per[0]);
                    if (x < 0) continue;
                    if (!inside(h, b, x, y, z)) continue;
                    long c = cell(h, x, y, z);
                    if (bid[c] >= 0 && bid[c] != k)
                        return fail(h, REF_E_OVERLAP, "two bodies cover the same cell");
                    bid[c] = (short)k;
                }
            }
        }
    }
    return REF_OK;
}

/* neighbour of cell (x,y,z) along direction a; -1 if it lies beyond a wall */
static long neighbour(const ref_lbm *h, int x, int y, int z, int a)
{
    int xn = wrap(x + EX[a], h->nx, h->bc & REF_BC_PERIODIC_X);
    int yn = wrap(y + EY[a], h->ny, h->bc & REF_BC_PERIODIC_Y);
    int zn = wrap(z + EZ[a], h->nz, h->bc & REF_BC_PERIODIC_Z);
    if (xn < 0 || yn < 0 || zn < 0) return -1;
    return cell(h, xn, yn, zn);
}

/* ---- step 2a: stream with bounce-back (Eq. 3, Eq. 4, moving-wall rule) --- */

static void stream(ref_lbm *h)
{
    const long C = h->C;
    const double *G = h->G;
    double *F = h->F;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < h->nz; ++z)
        for (int y = 0; y < h->ny; ++y)
            for (int x = 0; x < h->nx; ++x) {
                long c = cell(h, x, y, z);
                if (h->bid_prev[c] >= 0) continue;          /* obstacle at n-1 */
                double rho = 0.0;                            /* rho_w = sum f~ */
                for (int a = 0; a < Q; ++a) rho += G[a * C + c];
                F[0 * C + c] = G[0 * C + c];
                for (int a = 1; a < Q; ++a) {
                    long n = neighbour(h, x, y, z, a);
                    int ab = OPP[a];
                    if (n < 0) {
                        /* static no-slip wall, Eq. 4 */
                        F[ab * C + c] = G[a * C + c];
                    } else if (h->bid_prev[n] >= 0) {
                        /* moving obstacle: f_abar(x_f) = f~_a(x_f) + 6 w_a rho_w e_abar . u_w */
                        double p[3] = {x + EX[a], y + EY[a], z + EZ[a]}, uw[3];
                        wall_velocity(h, &h->body_prev[h->bid_prev[n]], p, uw);
                        double eu = EX[ab] * uw[0] + EY[ab] * uw[1] + EZ[ab] * uw[2];
                        F[ab * C + c] = G[a * C + c] + 6.0 * W[a] * rho * eu;
                    } else {
                        F[a * C + n] = G[a * C + c];
                    }
                }
            }
}

/* ---- step 2b: reconstruct uncovered cells (Sec. 2.3) -------------------- */

static void refill(ref_lbm *h)
{
    const long C = h->C;
    for (int z = 0; z < h->nz; ++z)
        for (int y = 0; y < h->ny; ++y)
            for (int x = 0; x < h->nx; ++x) {
                long c = cell(h, x, y, z);
                if (!(h->bid_prev[c] >= 0 && h->bid_now[c] < 0)) continue;
                double sum = 0.0;
                int cnt = 0;
                for (int a = 1; a < Q; ++a) {
                    long n = neighbour(h, x, y, z, a);
                    if (n < 0 || h->bid_prev[n] >= 0 || h->bid_now[n] >= 0) continue;
                    double rho = 0.0;
                    for (int b = 0; b < Q; ++b) rho += h->G[b * C + n];
                    sum += rho;
                    ++cnt;
                }
                double rho_avg = cnt ? sum / cnt : 1.0;
                double p[3] = {x, y, z}, uw[3];
                wall_velocity(h, &h->body[h->bid_prev[c]], p, uw);
                for (int a = 0; a < Q; ++a) h->F[a * C + c] = feq(a, rho_avg, uw);
            }
}

/* ---- step 2c: LBGK collision (Eq. 2) with Guo's body-force term ---------- */

static void collide(ref_lbm *h)
{
    const long C = h->C;
    const double tau = h->tau, *g = h->g;
    const int forced = g[0] != 0.0 || g[1] != 0.0 || g[2] != 0.0;
#pragma omp parallel for schedule(static)
    for (long c = 0; c < C; ++c) {
        if (h->bid_now[c] >= 0) {
            for (int a = 0; a < Q; ++a) h->G[a * C + c] = W[a];
            continue;
        }
        double rho = 0.0, m[3] = {0.0, 0.0, 0.0};
        for (int a = 0; a < Q; ++a) {
            double f = h->F[a * C + c];
            rho += f;
            m[0] += EX[a] * f; m[1] += EY[a] * f; m[2] += EZ[a] * f;
        }
        double u[3] = {(m[0] + 0.5 * g[0]) / rho, (m[1] + 0.5 * g[1]) / rho, (m[2] + 0.5 * g[2]) / rho};
        for (int a = 0; a < Q; ++a) {
            double f = h->F[a * C + c];
            double out = f - (f - feq(a, rho, u)) / tau;
            if (forced) {
                double eu = EX[a] * u[0] + EY[a] * u[1] + EZ[a] * u[2];
                double s = 3.0 * ((EX[a] - u[0]) * g[0] + (EY[a] - u[1]) * g[1] + (EZ[a] - u[2]) * g[2]) +
                           9.0 * eu * (EX[a] * g[0] + EY[a] * g[1] + EZ[a] * g[2]);
                out += (1.0 - 0.5 / tau) * W[a] * s;
            }
            h->G[a * C + c] = out;
        }
    }
}

/* ---- step 3: momentum-exchange force and torque (Eq. hydroF) ------------ */

/* Links (x_f, a) of body k: x_f fluid, x_f + e_a inside body k.  Every such
 * x_f lies in the body's bounding box grown by one cell, which is scanned in
 * z, y, x order (unwrapped box coordinates), then a = 1..18. */
static void hydro_force(ref_lbm *h)
{
    const long C = h->C;
    int per[3] = {h->bc & REF_BC_PERIODIC_X, h->bc & REF_BC_PERIODIC_Y, h->bc & REF_BC_PERIODIC_Z};
    memset(h->Fh, 0, sizeof h->Fh);
    memset(h->Th, 0, sizeof h->Th);
    for (int k = 0; k < h->nb; ++k) {
        const body_t *b = &h->body[k];
        double ext = b->r + 0.5 * b->l;
        int lo[3], hi[3], n[3] = {h->nx, h->ny, h->nz};
        for (int i = 0; i < 3; ++i) {
            lo[i] = (int)floor(b->X[i] - ext) - 2;
            hi[i] = (int)ceil(b->X[i] + ext) + 2;
            /* a periodic box wider than the domain would visit cells twice */
            if (per[i] && hi[i] - lo[i] + 1 > n[i]) { lo[i] = 0; hi[i] = n[i] - 1; }
        }
        for (int iz = lo[2]; iz <= hi[2]; ++iz) {
            int z = wrap(iz, h->nz, per[2]);
            if (z < 0) continue;
            for (int iy = lo[1]; iy <= hi[1]; ++iy) {
                int y = wrap(iy, h->ny, per[1]);
                if (y < 0) continue;
                for (int ix = lo[0]; ix <= hi[0]; ++ix) {
                    int x = wrap(ix, h->nx, per[0]);
                    if (x < 0) continue;
                    long c = cell(h, x, y, z);
                    if (h->bid_now[c] >= 0) continue;
                    double rho = -1.0;
                    for (int a = 1; a < Q; ++a) {
                        long nb = neighbour(h, x, y, z, a);
                        if (nb < 0 || h->bid_now[nb] != k) continue;
                        if (rho < 0) {
                            rho = 0.0;
                            for (int q = 0; q < Q; ++q) rho += h->G[q * C + c];
                        }
                        int ab = OPP[a];
                        double p[3] = {x + EX[a], y + EY[a], z + EZ[a]}, uw[3];
                        wall_velocity(h, b, p, uw);
                        double eu = EX[ab] * uw[0] + EY[ab] * uw[1] + EZ[ab] * uw[2];
                        double mag = 2.0 * h->G[a * C + c] + 6.0 * W[a] * rho * eu;
                        double fl[3] = {EX[a] * mag, EY[a] * mag, EZ[a] * mag};
                        double mid[3] = {x + 0.5 * EX[a], y + 0.5 * EY[a], z + 0.5 * EZ[a]}, d[3], t[3];
                        body_offset(h, b, mid, d);
                        cross(d, fl, t);
                        for (int i = 0; i < 3; ++i) { h->Fh[k][i] += fl[i]; h->Th[k][i] += t[i]; }
                    }
                }
            }
        }
    }
}

/* ---- steps 4-5: drive, springs and the rigid-body time step ------------- */

static int integrate_bodies(ref_lbm *h)
{
    double Ftot[MAX_BODIES][3], Tq[MAX_BODIES][3];
    double t = (double)h->step;
    /* with REF_OPT_AVERAGE_FORCE the step takes the mean hydrodynamic load
     * of this step and the previous one (from the second step on) */
    const int avg = (h->options & REF_OPT_AVERAGE_FORCE) && h->step > 0;
    for (int k = 0; k < h->nb; ++k) {
        const body_t *b = &h->body[k];
        for (int i = 0; i < 3; ++i) {
            const double f = avg ? 0.5 * (h->Fh[k][i] + h->Fh_prev[k][i]) : h->Fh[k][i];
            Tq[k][i] = avg ? 0.5 * (h->Th[k][i] + h->Th_prev[k][i]) : h->Th[k][i];
            Ftot[k][i] = f + h->g[i] * b->volume;
        }
    }
    memcpy(h->Fh_prev, h->Fh, sizeof h->Fh);
    memcpy(h->Th_prev, h->Th, sizeof h->Th);
    /* driving forces of the cycling strategy (Eq. FB1-FB3) along body x */
    for (int d = 0; d < h->nd; ++d) {
        const drive_t *dr = &h->drive[d];
        double omega = 2.0 * M_PI * dr->freq;
        if (t < dr->phase / omega || t >= dr->t_off) continue;
        double R[3][3];
        rot_matrix(h->body[dr->body].q, R);
        double f = dr->amp * sin(omega * t - dr->phase);
        /* the drive direction is a body-frame axis (default the body x axis) */
        for (int i = 0; i < 3; ++i)
            Ftot[dr->body][i] += f * (R[i][0] * dr->axis[0] + R[i][1] * dr->axis[1] + R[i][2] * dr->axis[2]);
    }
    /* damped harmonic springs (Eq. spring_i, damp_i, osci_i, osci_j) */
    for (int s = 0; s < h->ns; ++s) {
        const spring_t *sp = &h->spring[s];
        const body_t *bi = &h->body[sp->i], *bj = &h->body[sp->j];
        double d[3] = {bi->X[0] - bj->X[0], bi->X[1] - bj->X[1], bi->X[2] - bj->X[2]};
        double len = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        for (int i = 0; i < 3; ++i) {
            double dir = len > 0 ? d[i] / len : 0.0;
            double fi = -sp->k * (len - sp->rest) * dir - sp->gamma * (bi->V[i] - bj->V[i]);
            Ftot[sp->i][i] += fi;
            Ftot[sp->j][i] -= fi;
        }
    }
    /* Algorithm 1, time integration: semi-implicit Euler, dt = 1 */
    for (int k = 0; k < h->nb; ++k) {
        body_t *b = &h->body[k];
        h->body_prev[k] = *b;
        for (int i = 0; i < 3; ++i) {
            b->V[i] += Ftot[k][i] / b->m;
            b->X[i] += b->V[i];
        }
        /* Omega += I_world^-1 T with I_world^-1 = R diag(1/I) R^T */
        double R[3][3], Tb[3], dW[3];
        rot_matrix(b->q, R);
        for (int i = 0; i < 3; ++i)
            Tb[i] = R[0][i] * Tq[k][0] + R[1][i] * Tq[k][1] + R[2][i] * Tq[k][2];
        for (int i = 0; i < 3; ++i) Tb[i] /= b->inertia[i];
        for (int i = 0; i < 3; ++i) dW[i] = R[i][0] * Tb[0] + R[i][1] * Tb[1] + R[i][2] * Tb[2];
        for (int i = 0; i < 3; ++i) b->Om[i] += dW[i];
        /* q += 1/2 (0, Omega) (x) q, then renormalise */
        double w = b->q[0], v[3] = {b->q[1], b->q[2], b->q[3]}, c[3];
        cross(b->Om, v, c);
        double dq[4] = {-0.5 * (b->Om[0] * v[0] + b->Om[1] * v[1] + b->Om[2] * v[2]),
                        0.5 * (w * b->Om[0] + c[0]),
                        0.5 * (w * b->Om[1] + c[1]),
                        0.5 * (w * b->Om[2] + c[2])};
        double nn = 0.0;
        for (int i = 0; i < 4; ++i) { b->q[i] += dq[i]; nn += b->q[i] * b->q[i]; }
        nn = sqrt(nn);
        for (int i = 0; i < 4; ++i) b->q[i] /= nn;
        for (int i = 0; i < 3; ++i)
            if (!isfinite(b->X[i]) || !isfinite(b->V[i]) || !isfinite(b->Om[i]))
                return fail(h, REF_E_NAN, "non-finite body state");
    }
    return REF_OK;
}

/* ---- recording for the reverse sweep ------------------------------------ */

/* Everything the reverse sweep reads, for each recorded step j (forward step
 * n = t0 + j): the post-collision populations entering the step (G^{n-1}),
 * the pre-collision populations it forms (stream + refill), the obstacle
 * map of epoch n-1, the body states n-1 and n and the hydrodynamic force and
 * torque of the step.  Index n of Gin and bid holds the final ones, index
 * n + 1 of state the final body states. */
struct tape {
    int n, cap;
    long t0;
    double *Gin, *Fpre, *fh;
    short *bid;
    body_t *state;
};

/* FNV-1a digest of the obstacle map of a step, folded into a running value */
static unsigned long long digest_map(unsigned long long d, const short *bid, long C)
{
    if (d == 0) d = 1469598103934665603ULL;
    for (long c = 0; c < C; ++c) {
        d ^= (unsigned long long)(unsigned short)bid[c];
        d *= 1099511628211ULL;
    }
    return d;
}

/* ---- one coupled step (Algorithm 2) ------------------------------------- */

static int one_step(ref_lbm *h)
{
    if (!h->started) {
        /* the flag field before the first step equals the first mapping and
         * the bodies start from their given state */
        int rc = map_bodies(h, h->bid_prev);
        if (rc) return rc;
        for (int k = 0; k < h->nb; ++k) h->body_prev[k] = h->body[k];
        h->started = 1;
    }
    struct tape *tp = h->tape;
    const long QC = (long)Q * h->C;
    int rc = map_bodies(h, h->bid_now);             /* 1. map */
    if (rc) return rc;
    h->flag_digest = digest_map(h->flag_digest, h->bid_now, h->C);
    if (tp) {
        const int j = tp->n;
        memcpy(tp->Gin + j * QC, h->G, sizeof(double) * QC);
        memcpy(tp->bid + j * h->C, h->bid_prev, sizeof(short) * h->C);
        memcpy(tp->state + (long)j * h->nb, h->body_prev, sizeof(body_t) * h->nb);
        memcpy(tp->state + (long)(j + 1) * h->nb, h->body, sizeof(body_t) * h->nb);
    }
    stream(h);                                       /* 2. stream + bounce-back */
    refill(h);                                       /*    uncovered cells */
    if (tp) memcpy(tp->Fpre + tp->n * QC, h->F, sizeof(double) * QC);
    collide(h);                                      /*    LBGK */
    hydro_force(h);                                  /* 3. F_hydro, T_hydro */
    if (tp) {
        double *f = tp->fh + (long)tp->n * h->nb * 6;
        for (int k = 0; k < h->nb; ++k)
            for (int i = 0; i < 3; ++i) { f[6 * k + i] = h->Fh[k][i]; f[6 * k + 3 + i] = h->Th[k][i]; }
    }
    rc = integrate_bodies(h);                        /* 4.-5. drive, springs, pe */
    if (rc) return rc;
    short *t = h->bid_prev; h->bid_prev = h->bid_now; h->bid_now = t;
    h->step++;
    if (tp) tp->n++;
    if (h->avg_on) {                                 /* running velocity average (Sec. 6) */
        for (long c = 0; c < h->C; ++c) {
            double u[3];
            cell_velocity(h, c, h->bid_prev[c] >= 0, u);
            for (int i = 0; i < 3; ++i) h->avg_sum[i * h->C + c] += u[i];
        }
        h->avg_steps++;
    }
    return REF_OK;
}

/* Time average of the velocity field (Sec. 6, the flow fields averaged over
 * five swimming cycles): from the next step on, each step adds the velocity
 * of every cell after it (the REF_FIELD_U value) to a running sum. */
int lbm_ref_average_begin(ref_lbm *h)
{
    if (!h) return REF_E_ARG;
    if (!h->avg_sum) {
        h->avg_sum = malloc(sizeof(double) * 3 * h->C);
        if (!h->avg_sum) return fail(h, REF_E_OOM, "out of memory");
    }
    memset(h->avg_sum, 0, sizeof(double) * 3 * h->C);
    h->avg_steps = 0;
    h->avg_on = 1;
    return REF_OK;
}

/* the mean velocity [3][C] over the steps since lbm_ref_average_begin */
int lbm_ref_average_get(ref_lbm *h, double *out, long *steps)
{
    if (!h || !out || !h->avg_sum) return REF_E_ARG;
    for (long k = 0; k < 3 * h->C; ++k) out[k] = h->avg_steps ? h->avg_sum[k] / h->avg_steps : 0.0;
    if (steps) *steps = h->avg_steps;
    return REF_OK;
}

int lbm_ref_step(ref_lbm *h, int n)
{
    if (!h || n < 0) return REF_E_ARG;
    for (int i = 0; i < n; ++i) {
        int rc = one_step(h);
        if (rc) return rc;
    }
    return REF_OK;
}

/* ---- exports ------------------------------------------------------------ */

int lbm_ref_get_bodies(ref_lbm *h, double *out)
{
    if (!h || !out) return REF_E_ARG;
    for (int k = 0; k < h->nb; ++k) {
        const body_t *b = &h->body[k];
        double *o = out + 13 * k;
        for (int i = 0; i < 3; ++i) { o[i] = b->X[i]; o[7 + i] = b->V[i]; o[10 + i] = b->Om[i]; }
        for (int i = 0; i < 4; ++i) o[3 + i] = b->q[i];
    }
    return REF_OK;
}

int lbm_ref_get_forces(ref_lbm *h, double *out)
{
    if (!h || !out) return REF_E_ARG;
    for (int k = 0; k < h->nb; ++k)
        for (int i = 0; i < 3; ++i) { out[6 * k + i] = h->Fh[k][i]; out[6 * k + 3 + i] = h->Th[k][i]; }
    return REF_OK;
}

/* Fields of the last completed step: density rho = sum f~, velocity
 * u = (sum e f~ - g/2) / rho (the pre-collision velocity of Guo's scheme);
 * obstacle cells report rho = 1 and u = 0. */
int lbm_ref_get_fields(ref_lbm *h, int what, void *out)
{
    if (!h || !out) return REF_E_ARG;
    const long C = h->C;
    const short *bid = h->bid_prev;    /* flags of the last completed step */
    if (what == REF_FIELD_POP) {
        memcpy(out, h->G, sizeof(double) * Q * C);
        return REF_OK;
    }
    if (what == REF_FIELD_FLAGS) {
        unsigned char *o = out;
        for (long c = 0; c < C; ++c) o[c] = bid[c] >= 0 ? (unsigned char)(bid[c] + 1) : 0;
        return REF_OK;
    }
    if (what != REF_FIELD_RHO && what != REF_FIELD_U) return REF_E_ARG;
    double *o = out;
#pragma omp parallel for schedule(static)
    for (long c = 0; c < C; ++c) {
        double u[3];
        double rho = cell_velocity(h, c, bid[c] >= 0, u);
        if (what == REF_FIELD_RHO) {
            o[c] = rho;
        } else {
            for (int i = 0; i < 3; ++i) o[i * C + c] = u[i];
        }
    }
    return REF_OK;
}

/* Test hooks: the velocity set, the weights and the equilibrium function the
 * oracle uses, so that tests can check them against the closed-form moments
 * of the D3Q19 lattice. */
int lbm_ref_lattice(int *e, double *w)
{
    for (int a = 0; a < Q; ++a) {
        e[3 * a] = EX[a]; e[3 * a + 1] = EY[a]; e[3 * a + 2] = EZ[a];
        w[a] = W[a];
    }
    return Q;
}

int lbm_ref_equilibrium(double rho, const double u[3], double *out)
{
    for (int a = 0; a < Q; ++a) out[a] = feq(a, rho, u);
    return REF_OK;
}

/* Test hook: volume and principal moments of inertia of body b. */
int lbm_ref_body_props(ref_lbm *h, int b, double *out)
{
    if (!h || !out || b < 0 || b >= h->nb) return REF_E_ARG;
    out[0] = h->body[b].volume;
    for (int i = 0; i < 3; ++i) out[1 + i] = h->body[b].inertia[i];
    return REF_OK;
}

long lbm_ref_steps_done(ref_lbm *h) { return h ? h->step : -1; }

int lbm_ref_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* threads of the parallel loops from now on (n >= 1); returns the count in use */
int lbm_ref_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
    return lbm_ref_num_threads();
}

const char *lbm_ref_last_error(ref_lbm *h) { return h ? h->err : "null handle"; }

/* ==========================================================================
 * Reverse mode.  The gradient of J = sum_b seed_b . S_b(n0 + n), a linear
 * function of the body states after n steps, with respect to the drive
 * amplitudes and phases, the spring constants, rest lengths and dampings,
 * the body masses, principal moments of inertia and volumes, and the body
 * states and populations the run starts from.
 *
 * The obstacle maps of the recorded run are held fixed (the cell-centre test
 * of Sec. 2.3 is piecewise constant in the body positions), so J is the
 * smooth function of the parameters that the recorded map sequence defines.
 * The sweep applies, step by step in reverse, the transposed Jacobian of
 * each part of the step in reverse order: rigid-body step, momentum-exchange
 * force, collision, refill, stream with bounce-back.  The recording keeps
 * every step (no checkpoints): this is the plain version.
 * ========================================================================== */

/* adjoint of the surface velocity u_w = V + Omega x (p - X) of body b, for
 * the scalar uh . u_w: adds to the adjoint sa[13] of the body state */
static void adj_surface_velocity(const ref_lbm *h, const body_t *b, const double p[3], const double uh[3],
                                 double *sa)
{
    double o[3], c[3];
    body_offset(h, b, p, o);
    for (int i = 0; i < 3; ++i) sa[7 + i] += uh[i];
    cross(o, uh, c);                       /* uh . (Om x o) = Om . (o x uh) */
    for (int i = 0; i < 3; ++i) sa[10 + i] += c[i];
    cross(b->Om, uh, c);                   /* d/dX = -(uh x Om) = Om x uh */
    for (int i = 0; i < 3; ++i) sa[i] += c[i];
}

/* adjoint of R(q) (rot_matrix): qh += sum_ij Rh_ij dR_ij/dq */
static void adj_rot_matrix(const double q[4], const double Rh[3][3], double qh[4])
{
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    qh[2] += -4 * y * Rh[0][0]; qh[3] += -4 * z * Rh[0][0];
    qh[1] += 2 * y * Rh[0][1]; qh[2] += 2 * x * Rh[0][1]; qh[0] += -2 * z * Rh[0][1]; qh[3] += -2 * w * Rh[0][1];
    qh[1] += 2 * z * Rh[0][2]; qh[3] += 2 * x * Rh[0][2]; qh[0] += 2 * y * Rh[0][2]; qh[2] += 2 * w * Rh[0][2];
    qh[1] += 2 * y * Rh[1][0]; qh[2] += 2 * x * Rh[1][0]; qh[0] += 2 * z * Rh[1][0]; qh[3] += 2 * w * Rh[1][0];
    qh[1] += -4 * x * Rh[1][1]; qh[3] += -4 * z * Rh[1][1];
    qh[2] += 2 * z * Rh[1][2]; qh[3] += 2 * y * Rh[1][2]; qh[0] += -2 * x * Rh[1][2]; qh[1] += -2 * w * Rh[1][2];
    qh[1] += 2 * z * Rh[2][0]; qh[3] += 2 * x * Rh[2][0]; qh[0] += -2 * y * Rh[2][0]; qh[2] += -2 * w * Rh[2][0];
    qh[2] += 2 * z * Rh[2][1]; qh[3] += 2 * y * Rh[2][1]; qh[0] += 2 * x * Rh[2][1]; qh[1] += 2 * w * Rh[2][1];
    qh[1] += -4 * x * Rh[2][2]; qh[2] += -4 * y * Rh[2][2];
}

/* Reverse of integrate_bodies at step t from the states S (state n) and the
 * hydrodynamic loads fhyd (nb x 6).  Sn: adjoint of state n + 1 (input);
 * Sc: adjoint of state n (added to); Fa: adjoint of the hydrodynamic force
 * and torque (output); gd, gs, gb: parameter gradients (added to). */
static void integrate_adjoint(const ref_lbm *h, const body_t *S, const double *fhyd, long t,
                              const double (*Sn)[13], double (*Sc)[13], double (*Fa)[6],
                              double *gd, double *gs, double *gb)
{
    const int nb = h->nb;
    double (*Ftot)[3] = calloc(nb, sizeof *Ftot);
    double (*Fh)[3] = calloc(nb, sizeof *Fh);
    double (*Rh)[3][3] = calloc(nb, sizeof *Rh);
    /* the total force of the forward step, in the same order */
    for (int k = 0; k < nb; ++k)
        for (int i = 0; i < 3; ++i) Ftot[k][i] = fhyd[6 * k + i] + h->g[i] * S[k].volume;
    for (int d = 0; d < h->nd; ++d) {
        const drive_t *dr = &h->drive[d];
        double omega = 2.0 * M_PI * dr->freq;
        if ((double)t < dr->phase / omega || (double)t >= dr->t_off) continue;
        double R[3][3];
        rot_matrix(S[dr->body].q, R);
        double f = dr->amp * sin(omega * t - dr->phase);
        for (int i = 0; i < 3; ++i)
            Ftot[dr->body][i] += f * (R[i][0] * dr->axis[0] + R[i][1] * dr->axis[1] + R[i][2] * dr->axis[2]);
    }
    for (int s = 0; s < h->ns; ++s) {
        const spring_t *sp = &h->spring[s];
        const body_t *bi = &S[sp->i], *bj = &S[sp->j];
        double d[3] = {bi->X[0] - bj->X[0], bi->X[1] - bj->X[1], bi->X[2] - bj->X[2]};
        double len = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        for (int i = 0; i < 3; ++i) {
            double dir = len > 0 ? d[i] / len : 0.0;
            double fi = -sp->k * (len - sp->rest) * dir - sp->gamma * (bi->V[i] - bj->V[i]);
            Ftot[sp->i][i] += fi;
            Ftot[sp->j][i] -= fi;
        }
    }
    /* semi-implicit Euler, body by body */
    for (int k = 0; k < nb; ++k) {
        const body_t *b = &S[k];
        const double *sn = Sn[k];
        double R[3][3];
        rot_matrix(b->q, R);
        const double *T = fhyd + 6 * k + 3;
        double beta[3], Tb[3], Om1[3];
        for (int i = 0; i < 3; ++i) beta[i] = R[0][i] * T[0] + R[1][i] * T[1] + R[2][i] * T[2];
        for (int i = 0; i < 3; ++i) Tb[i] = beta[i] / b->inertia[i];
        for (int i = 0; i < 3; ++i) Om1[i] = b->Om[i] + R[i][0] * Tb[0] + R[i][1] * Tb[1] + R[i][2] * Tb[2];
        const double w = b->q[0], v[3] = {b->q[1], b->q[2], b->q[3]};
        double c[3];
        cross(Om1, v, c);
        double q4[4] = {w - 0.5 * (Om1[0] * v[0] + Om1[1] * v[1] + Om1[2] * v[2]),
                        v[0] + 0.5 * (w * Om1[0] + c[0]), v[1] + 0.5 * (w * Om1[1] + c[1]),
                        v[2] + 0.5 * (w * Om1[2] + c[2])};
        double nn = sqrt(q4[0] * q4[0] + q4[1] * q4[1] + q4[2] * q4[2] + q4[3] * q4[3]);
        double q1[4] = {q4[0] / nn, q4[1] / nn, q4[2] / nn, q4[3] / nn};
        /* q1 = q4 / |q4| */
        double dot = 0.0, qh4[4];
        for (int i = 0; i < 4; ++i) dot += q1[i] * sn[3 + i];
        for (int i = 0; i < 4; ++i) qh4[i] = (sn[3 + i] - q1[i] * dot) / nn;
        /* q4 = q + (0, Om1) (x) q / 2 */
        const double qv[3] = {qh4[1], qh4[2], qh4[3]};
        double t1[3], t2[3];
        Sc[k][3] += qh4[0] + 0.5 * (qv[0] * Om1[0] + qv[1] * Om1[1] + qv[2] * Om1[2]);
        cross(qv, Om1, t1);
        for (int i = 0; i < 3; ++i) Sc[k][4 + i] += qv[i] - 0.5 * qh4[0] * Om1[i] + 0.5 * t1[i];
        double Oh1[3];
        cross(v, qv, t2);
        for (int i = 0; i < 3; ++i) Oh1[i] = sn[10 + i] - 0.5 * qh4[0] * v[i] + 0.5 * w * qv[i] + 0.5 * t2[i];
        /* Om1 = Om + R diag(1/I) R^T T */
        double alpha[3];
        for (int i = 0; i < 3; ++i) alpha[i] = R[0][i] * Oh1[0] + R[1][i] * Oh1[1] + R[2][i] * Oh1[2];
        for (int i = 0; i < 3; ++i) {
            Sc[k][10 + i] += Oh1[i];
            Fa[k][3 + i] = R[i][0] * alpha[0] / b->inertia[0] + R[i][1] * alpha[1] / b->inertia[1] +
                           R[i][2] * alpha[2] / b->inertia[2];
            gb[5 * k + 1 + i] += -beta[i] * alpha[i] / (b->inertia[i] * b->inertia[i]);
        }
        for (int i = 0; i < 3; ++i)
            for (int jj = 0; jj < 3; ++jj)
                Rh[k][i][jj] += Oh1[i] * beta[jj] / b->inertia[jj] + T[i] * alpha[jj] / b->inertia[jj];
        /* X1 = X + V1, V1 = V + F / m */
        double Vh1[3], F2 = 0.0;
        for (int i = 0; i < 3; ++i) {
            Vh1[i] = sn[7 + i] + sn[i];
            Sc[k][i] += sn[i];
            Sc[k][7 + i] += Vh1[i];
            Fh[k][i] = Vh1[i] / b->m;
            Fa[k][i] = Fh[k][i];
            F2 += Vh1[i] * Ftot[k][i];
            gb[5 * k + 4] += h->g[i] * Fh[k][i];
        }
        gb[5 * k] += -F2 / (b->m * b->m);
    }
    /* drive terms */
    for (int d = 0; d < h->nd; ++d) {
        const drive_t *dr = &h->drive[d];
        double omega = 2.0 * M_PI * dr->freq;
        if ((double)t < dr->phase / omega || (double)t >= dr->t_off) continue;
        double R[3][3];
        rot_matrix(S[dr->body].q, R);
        const double sn_ = sin(omega * t - dr->phase), cs = cos(omega * t - dr->phase);
        const double *fh_ = Fh[dr->body], *a = dr->axis;
        double dir[3], proj = 0.0;
        for (int i = 0; i < 3; ++i) {
            dir[i] = R[i][0] * a[0] + R[i][1] * a[1] + R[i][2] * a[2];
            proj += fh_[i] * dir[i];
        }
        gd[2 * d] += sn_ * proj;
        gd[2 * d + 1] += -dr->amp * cs * proj;
        /* F = f R a: dF_i / dR_ij = f a_j */
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) Rh[dr->body][i][j] += dr->amp * sn_ * fh_[i] * a[j];
    }
    /* springs */
    for (int s = 0; s < h->ns; ++s) {
        const spring_t *sp = &h->spring[s];
        const body_t *bi = &S[sp->i], *bj = &S[sp->j];
        double d[3] = {bi->X[0] - bj->X[0], bi->X[1] - bj->X[1], bi->X[2] - bj->X[2]};
        double len = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        double fh_[3], dv = 0.0;
        for (int i = 0; i < 3; ++i) {
            fh_[i] = Fh[sp->i][i] - Fh[sp->j][i];
            dv += fh_[i] * (bi->V[i] - bj->V[i]);
            Sc[sp->i][7 + i] += -sp->gamma * fh_[i];
            Sc[sp->j][7 + i] += sp->gamma * fh_[i];
        }
        gs[3 * s + 2] += -dv;
        if (!(len > 0)) continue;
        double dir[3] = {d[0] / len, d[1] / len, d[2] / len};
        double fd = fh_[0] * dir[0] + fh_[1] * dir[1] + fh_[2] * dir[2];
        gs[3 * s] += -(len - sp->rest) * fd;
        gs[3 * s + 1] += sp->k * fd;
        for (int i = 0; i < 3; ++i) {
            double da = -sp->k * (fd * dir[i] + (len - sp->rest) / len * (fh_[i] - fd * dir[i]));
            Sc[sp->i][i] += da;
            Sc[sp->j][i] -= da;
        }
    }
    for (int k = 0; k < nb; ++k) adj_rot_matrix(S[k].q, Rh[k], Sc[k] + 3);
    free(Ftot); free(Fh); free(Rh);
}

/* Reverse of hydro_force for the populations G (step n), map bid and body
 * states S of step n: adds to Ga (adjoint of G) and Sc (adjoint of S). */
static void hydro_force_adjoint(const ref_lbm *h, const double *G, const short *bid, const body_t *S,
                                const double (*Fa)[6], double *Ga, double (*Sc)[13])
{
    const long C = h->C;
    int per[3] = {h->bc & REF_BC_PERIODIC_X, h->bc & REF_BC_PERIODIC_Y, h->bc & REF_BC_PERIODIC_Z};
    for (int k = 0; k < h->nb; ++k) {
        const body_t *b = &S[k];
        const double *Fk = Fa[k], *Tk = Fa[k] + 3;
        double ext = b->r + 0.5 * b->l;
        int lo[3], hi[3], n[3] = {h->nx, h->ny, h->nz};
        for (int i = 0; i < 3; ++i) {
            lo[i] = (int)floor(b->X[i] - ext) - 2;
            hi[i] = (int)ceil(b->X[i] + ext) + 2;
            if (per[i] && hi[i] - lo[i] + 1 > n[i]) { lo[i] = 0; hi[i] = n[i] - 1; }
        }
        for (int iz = lo[2]; iz <= hi[2]; ++iz) {
            int z = wrap(iz, h->nz, per[2]);
            if (z < 0) continue;
            for (int iy = lo[1]; iy <= hi[1]; ++iy) {
                int y = wrap(iy, h->ny, per[1]);
                if (y < 0) continue;
                for (int ix = lo[0]; ix <= hi[0]; ++ix) {
                    int x = wrap(ix, h->nx, per[0]);
                    if (x < 0) continue;
                    long c = cell(h, x, y, z);
                    if (bid[c] >= 0) continue;
                    double rho = 0.0;
                    for (int q = 0; q < Q; ++q) rho += G[q * C + c];
                    for (int a = 1; a < Q; ++a) {
                        long nbr = neighbour(h, x, y, z, a);
                        if (nbr < 0 || bid[nbr] != k) continue;
                        int ab = OPP[a];
                        double p[3] = {x + EX[a], y + EY[a], z + EZ[a]}, uw[3];
                        wall_velocity(h, b, p, uw);
                        double eu = EX[ab] * uw[0] + EY[ab] * uw[1] + EZ[ab] * uw[2];
                        double mag = 2.0 * G[a * C + c] + 6.0 * W[a] * rho * eu;
                        double e[3] = {EX[a], EY[a], EZ[a]};
                        double mid[3] = {x + 0.5 * EX[a], y + 0.5 * EY[a], z + 0.5 * EZ[a]}, d[3], de[3];
                        body_offset(h, b, mid, d);
                        cross(d, e, de);
                        /* F_link = e mag, T_link = d x e mag */
                        double mh = e[0] * Fk[0] + e[1] * Fk[1] + e[2] * Fk[2] +
                                    de[0] * Tk[0] + de[1] * Tk[1] + de[2] * Tk[2];
                        Ga[a * C + c] += 2.0 * mh;
                        for (int q = 0; q < Q; ++q) Ga[q * C + c] += 6.0 * W[a] * eu * mh;
                        double s = 6.0 * W[a] * rho * mh;
                        double uh[3] = {EX[ab] * s, EY[ab] * s, EZ[ab] * s};
                        adj_surface_velocity(h, b, p, uh, Sc[k]);
                        /* the lever arm d = mid - X: Xh += Th x F_link */
                        double fl[3] = {e[0] * mag, e[1] * mag, e[2] * mag}, tf[3];
                        cross(Tk, fl, tf);
                        for (int i = 0; i < 3; ++i) Sc[k][i] += tf[i];
                    }
                }
            }
        }
    }
}

/* Reverse of the LBGK collision with Guo's term at one cell: f holds the
 * pre-collision populations, gh the adjoint of the post-collision ones. */
static void collide_adjoint_cell(const ref_lbm *h, const double *f, const double *gh, double *fh)
{
    const double tau = h->tau, *g = h->g, om = 1.0 / tau;
    const int forced = g[0] != 0.0 || g[1] != 0.0 || g[2] != 0.0;
    double rho = 0.0, m[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < Q; ++a) {
        rho += f[a];
        m[0] += EX[a] * f[a]; m[1] += EY[a] * f[a]; m[2] += EZ[a] * f[a];
    }
    double u[3] = {(m[0] + 0.5 * g[0]) / rho, (m[1] + 0.5 * g[1]) / rho, (m[2] + 0.5 * g[2]) / rho};
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    double sr = 0.0, su[3] = {0.0, 0.0, 0.0};
    for (int b = 0; b < Q; ++b) {
        double e[3] = {EX[b], EY[b], EZ[b]};
        double eu = e[0] * u[0] + e[1] * u[1] + e[2] * u[2];
        sr += gh[b] * om * W[b] * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
        for (int i = 0; i < 3; ++i) su[i] += gh[b] * om * W[b] * rho * (3.0 * e[i] + 9.0 * eu * e[i] - 3.0 * u[i]);
        if (forced) {
            double eg = e[0] * g[0] + e[1] * g[1] + e[2] * g[2];
            for (int i = 0; i < 3; ++i) su[i] += gh[b] * (1.0 - 0.5 / tau) * W[b] * (-3.0 * g[i] + 9.0 * e[i] * eg);
        }
    }
    for (int a = 0; a < Q; ++a) {
        double e[3] = {EX[a], EY[a], EZ[a]};
        fh[a] = (1.0 - om) * gh[a] + sr;
        for (int i = 0; i < 3; ++i) fh[a] += su[i] * (e[i] - u[i]) / rho;
    }
}

/* Reverse of refill: Fa adjoint of the pre-collision populations of step n,
 * G the populations entering the step, bid_prev / bid_now the maps of epochs
 * n-1 and n, S the body states of step n.  Adds to Gp (adjoint of G) and Sc. */
static void refill_adjoint(const ref_lbm *h, const double *Fa, const double *G, const short *bid_prev,
                           const short *bid_now, const body_t *S, double *Gp, double (*Sc)[13])
{
    const long C = h->C;
    for (int z = 0; z < h->nz; ++z)
        for (int y = 0; y < h->ny; ++y)
            for (int x = 0; x < h->nx; ++x) {
                long c = cell(h, x, y, z);
                if (!(bid_prev[c] >= 0 && bid_now[c] < 0)) continue;
                double sum = 0.0;
                int cnt = 0;
                for (int a = 1; a < Q; ++a) {
                    long n = neighbour(h, x, y, z, a);
                    if (n < 0 || bid_prev[n] >= 0 || bid_now[n] >= 0) continue;
                    for (int b = 0; b < Q; ++b) sum += G[b * C + n];
                    ++cnt;
                }
                double rho_avg = cnt ? sum / cnt : 1.0;
                const body_t *b = &S[bid_prev[c]];
                double p[3] = {x, y, z}, uw[3];
                wall_velocity(h, b, p, uw);
                double uu = uw[0] * uw[0] + uw[1] * uw[1] + uw[2] * uw[2];
                double rh = 0.0, uh[3] = {0.0, 0.0, 0.0};
                for (int a = 0; a < Q; ++a) {
                    double e[3] = {EX[a], EY[a], EZ[a]};
                    double eu = e[0] * uw[0] + e[1] * uw[1] + e[2] * uw[2];
                    double fa = Fa[a * C + c];
                    rh += fa * W[a] * (1.0 + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
                    for (int i = 0; i < 3; ++i) uh[i] += fa * W[a] * rho_avg * (3.0 * e[i] + 9.0 * eu * e[i] - 3.0 * uw[i]);
                }
                if (cnt) {
                    for (int a = 1; a < Q; ++a) {
                        long n = neighbour(h, x, y, z, a);
                        if (n < 0 || bid_prev[n] >= 0 || bid_now[n] >= 0) continue;
                        for (int q = 0; q < Q; ++q) Gp[q * C + n] += rh / cnt;
                    }
                }
                adj_surface_velocity(h, b, p, uh, Sc[bid_prev[c]]);
            }
}

/* Reverse of stream: Fa adjoint of the pre-collision populations of step n,
 * G the populations entering the step, bid_prev the map of epoch n-1, Sp
 * the body states n-1.  Adds to Gp (adjoint of G) and Spa (adjoint of Sp). */
static void stream_adjoint(const ref_lbm *h, const double *Fa, const double *G, const short *bid_prev,
                           const body_t *Sp, double *Gp, double (*Spa)[13])
{
    const long C = h->C;
    for (int z = 0; z < h->nz; ++z)
        for (int y = 0; y < h->ny; ++y)
            for (int x = 0; x < h->nx; ++x) {
                long c = cell(h, x, y, z);
                if (bid_prev[c] >= 0) continue;
                double rho = 0.0;
                for (int a = 0; a < Q; ++a) rho += G[a * C + c];
                double cr = 0.0;
                Gp[0 * C + c] += Fa[0 * C + c];
                for (int a = 1; a < Q; ++a) {
                    long n = neighbour(h, x, y, z, a);
                    int ab = OPP[a];
                    if (n < 0) {
                        Gp[a * C + c] += Fa[ab * C + c];
                    } else if (bid_prev[n] >= 0) {
                        const body_t *b = &Sp[bid_prev[n]];
                        double p[3] = {x + EX[a], y + EY[a], z + EZ[a]}, uw[3];
                        wall_velocity(h, b, p, uw);
                        double eu = EX[ab] * uw[0] + EY[ab] * uw[1] + EZ[ab] * uw[2];
                        double fa = Fa[ab * C + c];
                        Gp[a * C + c] += fa;
                        cr += 6.0 * W[a] * eu * fa;
                        double s = 6.0 * W[a] * rho * fa;
                        double uh[3] = {EX[ab] * s, EY[ab] * s, EZ[ab] * s};
                        adj_surface_velocity(h, b, p, uh, Spa[bid_prev[n]]);
                    } else {
                        Gp[a * C + c] += Fa[a * C + n];
                    }
                }
                for (int q = 0; q < Q; ++q) Gp[q * C + c] += cr;
            }
}

static void free_tape(struct tape *tp)
{
    if (!tp) return;
    free(tp->Gin); free(tp->Fpre); free(tp->fh); free(tp->bid); free(tp->state);
    free(tp);
}

int lbm_ref_adjoint(ref_lbm *h, int n, const double *seed, double *grad_state, double *grad_prev,
                    double *grad_pop, double *grad_drive, double *grad_spring, double *grad_body)
{
    if (!h || n < 1 || !seed) return REF_E_ARG;
    if (h->options & REF_OPT_AVERAGE_FORCE) return fail(h, REF_E_ARG, "no reverse mode with the averaged load");
    const long C = h->C, QC = (long)Q * C;
    const int nb = h->nb;
    const int first_run = !h->started;
    struct tape *tp = calloc(1, sizeof *tp);
    if (!tp) return REF_E_OOM;
    tp->cap = n;
    tp->t0 = h->step;
    tp->Gin = malloc(sizeof(double) * (size_t)(n + 1) * QC);
    tp->Fpre = malloc(sizeof(double) * (size_t)n * QC);
    tp->fh = malloc(sizeof(double) * (size_t)n * (nb ? nb : 1) * 6);
    tp->bid = malloc(sizeof(short) * (size_t)(n + 1) * C);
    tp->state = malloc(sizeof(body_t) * (size_t)(n + 2) * (nb ? nb : 1));
    if (!tp->Gin || !tp->Fpre || !tp->fh || !tp->bid || !tp->state) {
        free_tape(tp);
        return REF_E_OOM;
    }
    /* forward, recorded */
    h->tape = tp;
    int rc = lbm_ref_step(h, n);
    h->tape = NULL;
    if (rc) { free_tape(tp); return rc; }
    memcpy(tp->Gin + (long)n * QC, h->G, sizeof(double) * QC);
    memcpy(tp->bid + (long)n * C, h->bid_prev, sizeof(short) * C);
    memcpy(tp->state + (long)(n + 1) * nb, h->body, sizeof(body_t) * nb);

    double *Ga = calloc(QC, sizeof(double));      /* adjoint of G^n */
    double *Gp = calloc(QC, sizeof(double));      /* adjoint of G^{n-1} */
    double *Fa = calloc(QC, sizeof(double));      /* adjoint of the pre-collision populations */
    double (*Sn)[13] = calloc(nb ? nb : 1, sizeof *Sn);   /* adjoint of state n + 1 */
    double (*Sc)[13] = calloc(nb ? nb : 1, sizeof *Sc);   /* adjoint of state n */
    double (*Sq)[13] = calloc(nb ? nb : 1, sizeof *Sq);   /* adjoint of state n - 1 (bounce-back) */
    double (*Fh)[6] = calloc(nb ? nb : 1, sizeof *Fh);
    double *gd = calloc(2 * (h->nd ? h->nd : 1), sizeof(double));
    double *gs = calloc(3 * (h->ns ? h->ns : 1), sizeof(double));
    double *gb = calloc(5 * (nb ? nb : 1), sizeof(double));
    if (!Ga || !Gp || !Fa || !Sn || !Sc || !Sq || !Fh || !gd || !gs || !gb) {
        rc = REF_E_OOM;
        goto done;
    }
    for (int k = 0; k < nb; ++k)
        for (int i = 0; i < 13; ++i) Sn[k][i] = seed[13 * k + i];
    const int with_fluid = !(h->options & REF_OPT_NO_FLUID);
    for (int j = n - 1; j >= 0; --j) {
        const body_t *Sprev = tp->state + (long)j * nb, *Scur = tp->state + (long)(j + 1) * nb;
        const double *Gin = tp->Gin + (long)j * QC, *Gout = tp->Gin + (long)(j + 1) * QC;
        const double *Fpre = tp->Fpre + (long)j * QC;
        const short *bprev = tp->bid + (long)j * C, *bnow = tp->bid + (long)(j + 1) * C;
        /* Sc starts with the bounce-back terms of step n + 1 (held in Sq) */
        memcpy(Sc, Sq, sizeof(double) * 13 * nb);
        integrate_adjoint(h, Scur, tp->fh + (long)j * nb * 6, tp->t0 + j, (const double (*)[13])Sn, Sc, Fh,
                          gd, gs, gb);
        memset(Sq, 0, sizeof(double) * 13 * nb);
        memset(Gp, 0, sizeof(double) * QC);
        if (with_fluid) {
            hydro_force_adjoint(h, Gout, bnow, Scur, (const double (*)[6])Fh, Ga, Sc);
            for (long c = 0; c < C; ++c) {
                double f[Q], gh[Q], fh[Q];
                if (bnow[c] >= 0) {
                    for (int a = 0; a < Q; ++a) Fa[a * C + c] = 0.0;
                    continue;
                }
                for (int a = 0; a < Q; ++a) { f[a] = Fpre[a * C + c]; gh[a] = Ga[a * C + c]; }
                collide_adjoint_cell(h, f, gh, fh);
                for (int a = 0; a < Q; ++a) Fa[a * C + c] = fh[a];
            }
            refill_adjoint(h, Fa, Gin, bprev, bnow, Scur, Gp, Sc);
            stream_adjoint(h, Fa, Gin, bprev, Sprev, Gp, Sq);
        }
        memcpy(Sn, Sc, sizeof(double) * 13 * nb);
        double *t = Ga; Ga = Gp; Gp = t;
    }
    /* Sn: adjoint of the first state; Sq: of the state before it, which is
     * the same state when the run began at the very first step */
    if (first_run)
        for (int k = 0; k < nb; ++k)
            for (int i = 0; i < 13; ++i) { Sn[k][i] += Sq[k][i]; Sq[k][i] = 0.0; }
    if (grad_state) memcpy(grad_state, Sn, sizeof(double) * 13 * nb);
    if (grad_prev) memcpy(grad_prev, Sq, sizeof(double) * 13 * nb);
    if (grad_pop) memcpy(grad_pop, Ga, sizeof(double) * QC);
    if (grad_drive) memcpy(grad_drive, gd, sizeof(double) * 2 * h->nd);
    if (grad_spring) memcpy(grad_spring, gs, sizeof(double) * 3 * h->ns);
    if (grad_body) memcpy(grad_body, gb, sizeof(double) * 5 * nb);
    rc = REF_OK;
done:
    free(Ga); free(Gp); free(Fa); free(Sn); free(Sc); free(Sq); free(Fh); free(gd); free(gs); free(gb);
    free_tape(tp);
    return rc;
}

unsigned long long lbm_ref_flag_digest(ref_lbm *h) { return h ? h->flag_digest : 0; }

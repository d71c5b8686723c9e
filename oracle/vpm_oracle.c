/*
 * FP64 CPU oracle of the vortex particle model (VPM) glider rollouts and MPPI reweighting of
 * "Real-Time Maneuver Planning for Fixed-Wing UAVs in Unsteady Flows Using a GPU-Accelerated
 * Vortex Particle Model" (§III-A, §III-B, §IV-A).
 *
 * TEST INFRASTRUCTURE. Only the tests, the smoke check and the benchmark's CPU-baseline leg
 * call this code. It shares no code with the CUDA library and never calls it. Every loop is
 * written plainly, in the order the paper states the model, with no blocking, fusion or
 * reordering, so that it can be checked against the paper by eye. Floating point is IEEE
 * binary64 with round-to-nearest (build without -ffast-math).
 *
 * Coordinates are (x, z), z up; e_z x (a, b) = (-b, a) and the planar cross product is
 * a x b = a_x b_z - a_z b_x, both counter-clockwise positive. Positive circulation is
 * counter-clockwise, positive pitch theta is nose-up.
 *
 * Readings of points the paper leaves open (each is a parameter or stated below):
 *  - the wing centre x_w is the "surface origin" r_g; the leading edge is the forward end,
 *    LE = x_w + (c/2)(cos th, sin th); e_t points from the LE to the TE; e_n = (-sin th, cos th)
 *    is the body-up normal, the same convention as the elevator normal of §III-B;
 *  - N_c = N_b + 1 collocation points at s_i = -c/2 + i c/N_b along e_t (LE first), bound
 *    vortices at the panel midpoints, l_b = c/N_b; LEV at LE - delta_s e_t, TEV at
 *    TE + delta_s e_t;
 *  - Eq. 12's relative velocity is taken as fluid minus surface-point velocity,
 *    sum K' Gamma + U_inf - v - omega e_z x (r_s - r_g) (the printed rotation term has the
 *    opposite sign);
 *  - M_w is the counter-clockwise moment about x_w of the pressure forces of Eq. 14,
 *    sum (r_b - x_w) x (l_b s dp e_n);
 *  - the time derivatives in Eq. 13 are backward differences over one step, zero on the
 *    first step. Every step sheds a new LEV (§III-A), and the potential jump across the
 *    plate at panel i holds the bound circulation from the leading edge to panel i plus all
 *    circulation shed at the leading edge so far. Its derivative therefore takes the new
 *    LEV's whole circulation over the step: dGamma_LEV/dt = Gamma_LEV^n / dt, the rate at
 *    which the leading edge sheds circulation;
 *  - the moment arms of §III-B's pitch equation are the world-frame offsets of x_w and x_e
 *    (Eq. 18) from the centre of gravity;
 *  - step order: geometry, relative velocity at the plate from the wake before shedding,
 *    surface solve, pressure and loads, append LEV/TEV, convection velocities of the enlarged
 *    wake, explicit Euler advection, decay Gamma <- Gamma exp(-gamma dt), glider Euler update,
 *    merging of the two oldest particles while N > N_w,max;
 *  - separation gate (§III-A): mode 1 sheds nothing while |alpha| <= alpha_crit, mode 2 sheds
 *    the TEV every step and the LEV only above alpha_crit; a collocation row at an edge that
 *    sheds nothing is dropped so the system stays square.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORA_MAXB 64
#define ORA_PI 3.14159265358979323846

enum { ORA_SINGULAR = 0, ORA_VATISTAS = 1, ORA_GAUSSIAN = 2 };
enum { ORA_OK = 0, ORA_ERR_CAPACITY = 3, ORA_ERR_SINGULAR = 8, ORA_ERR_INVALID = 1 };

typedef struct {
    int n_b;
    double chord, span, rho;
    int wake_kernel;
    double r_core;
    double shed_offset;     /* delta_s as a fraction of the chord */
    double gamma_decay;     /* gamma of Eq. 17 */
    int shed_gate;
    double alpha_crit;
    int n_wake_max;         /* 0: no merging */
    double u_inf_x, u_inf_z;
    double dt;
    int fixed_plate;        /* 1: the glider state is held fixed and the plate does not move */
    double mass, inertia, g, l, l_w, l_e, s_e;
    double q[7], x_d[7];
} ora_params;

/* ------------------------------------------------------------------ kernels (§III-A) */

/* Singular kernel of Eq. 4 for a unit circulation: K = -1/(2 pi r^2) J dr with
 * J = [[0, 1], [-1, 0]] and dr = r - r_v. Returns 0 at r = 0. */
static void kernel_singular(double dx, double dz, double *kx, double *kz)
{
    double r2 = dx * dx + dz * dz;
    if (r2 == 0.0) { *kx = 0.0; *kz = 0.0; return; }
    double jx = dz;     /* first row of J times dr  */
    double jz = -dx;    /* second row of J times dr */
    double s = -1.0 / (2.0 * ORA_PI * r2);
    *kx = s * jx;
    *kz = s * jz;
}

/* Core factor of Eq. 5: (r/r_core)^2 / sqrt(1 + (r/r_core)^4). */
static double factor_vatistas(double r, double rc)
{
    double q = (r / rc) * (r / rc);
    return q / sqrt(1.0 + q * q);
}

/* Gaussian core factor 1 - exp(-r^2 / delta^2). */
static double factor_gaussian(double r, double rc)
{
    return 1.0 - exp(-(r * r) / (rc * rc));
}

/* Kernel of the given kind for a unit circulation at displacement dr = r - r_v. */
static void kernel_eval(int kind, double rc, double dx, double dz, double *kx, double *kz)
{
    kernel_singular(dx, dz, kx, kz);
    if (kind == ORA_SINGULAR) return;
    double r = sqrt(dx * dx + dz * dz);
    double f = (kind == ORA_VATISTAS) ? factor_vatistas(r, rc) : factor_gaussian(r, rc);
    *kx *= f;
    *kz *= f;
}

void ora_kernel(int kind, double rc, double dx, double dz, double *kx, double *kz)
{
    kernel_eval(kind, rc, dx, dz, kx, kz);
}

/* Velocity at (tx, tz) of point vortices (Eq. 3): sum_v K_v(r) Gamma_v, skipping index `skip`. */
static void induced(int kind, double rc, int n, const double *x, const double *z, const double *g,
                    double tx, double tz, int skip, double *u, double *w)
{
    double su = 0.0, sw = 0.0;
    for (int v = 0; v < n; ++v) {
        if (v == skip) continue;
        double kx, kz;
        kernel_eval(kind, rc, tx - x[v], tz - z[v], &kx, &kz);
        su += kx * g[v];
        sw += kz * g[v];
    }
    *u = su;
    *w = sw;
}

/* Velocity of every particle of a free field from all the others (Eq. 16 without a plate). */
void ora_free_velocity(int n, const double *x, const double *z, const double *g, int kind,
                       double rc, double *u, double *w)
{
    for (int i = 0; i < n; ++i)
        induced(kind, rc, n, x, z, g, x[i], z[i], i, &u[i], &w[i]);
}

/* Velocity at m target points; skip[t] is the source index equal to target t (or -1). */
void ora_velocity_at(int n, const double *x, const double *z, const double *g, int kind, double rc,
                     int m, const double *tx, const double *tz, const long long *skip,
                     double *u, double *w)
{
    for (int t = 0; t < m; ++t)
        induced(kind, rc, n, x, z, g, tx[t], tz[t], skip ? (int)skip[t] : -1, &u[t], &w[t]);
}

/* Free-field explicit Euler: r <- r + dt v(r). */
void ora_free_euler(int n, double *x, double *z, const double *g, int kind, double rc, double dt,
                    int steps)
{
    double *u = malloc(sizeof(double) * n), *w = malloc(sizeof(double) * n);
    for (int s = 0; s < steps; ++s) {
        ora_free_velocity(n, x, z, g, kind, rc, u, w);
        for (int i = 0; i < n; ++i) { x[i] += dt * u[i]; z[i] += dt * w[i]; }
    }
    free(u); free(w);
}

/* Free-field Heun (explicit trapezoidal RK2): v1 = V(r); r* = r + dt v1; v2 = V(r*);
 * r <- r + dt/2 (v1 + v2). */
void ora_free_heun(int n, double *x, double *z, const double *g, int kind, double rc, double dt,
                   int steps)
{
    double *u1 = malloc(sizeof(double) * n), *w1 = malloc(sizeof(double) * n);
    double *u2 = malloc(sizeof(double) * n), *w2 = malloc(sizeof(double) * n);
    double *xs = malloc(sizeof(double) * n), *zs = malloc(sizeof(double) * n);
    for (int s = 0; s < steps; ++s) {
        ora_free_velocity(n, x, z, g, kind, rc, u1, w1);
        for (int i = 0; i < n; ++i) { xs[i] = x[i] + dt * u1[i]; zs[i] = z[i] + dt * w1[i]; }
        ora_free_velocity(n, xs, zs, g, kind, rc, u2, w2);
        for (int i = 0; i < n; ++i) {
            x[i] += 0.5 * dt * (u1[i] + u2[i]);
            z[i] += 0.5 * dt * (w1[i] + w2[i]);
        }
    }
    free(u1); free(w1); free(u2); free(w2); free(xs); free(zs);
}

/* ------------------------------------------------------------------ plate geometry */

typedef struct {
    int n_b, n_c;
    double lb;
    double xw, zw;              /* surface origin r_g = wing centre x_w */
    double tx, tz, nx, nz;      /* e_t (LE -> TE) and e_n */
    double vx, vz, omega;       /* plate velocity and angular velocity */
    double cx[ORA_MAXB + 1], cz[ORA_MAXB + 1];
    double bx[ORA_MAXB], bz[ORA_MAXB];
    double lev_x, lev_z, tev_x, tev_z;
} ora_geom;

/* Wing position and velocity from the glider state (§III-B, Eq. 18) and the plate points. */
static void plate_geometry(const ora_params *p, const double *xg, ora_geom *G)
{
    double th = xg[2], c = cos(th), s = sin(th);
    G->n_b = p->n_b;
    G->n_c = p->n_b + 1;
    G->lb = p->chord / p->n_b;
    G->xw = xg[0] - p->l_w * c;
    G->zw = xg[1] - p->l_w * s;
    G->tx = -c;  G->tz = -s;
    G->nx = -s;  G->nz = c;
    if (p->fixed_plate) {
        G->vx = 0.0; G->vz = 0.0; G->omega = 0.0;
    } else {
        G->vx = xg[4] + p->l_w * xg[6] * s;
        G->vz = xg[5] - p->l_w * xg[6] * c;
        G->omega = xg[6];
    }
    for (int i = 0; i < G->n_c; ++i) {
        double si = -0.5 * p->chord + i * G->lb;
        G->cx[i] = G->xw + si * G->tx;
        G->cz[i] = G->zw + si * G->tz;
    }
    for (int j = 0; j < G->n_b; ++j) {
        double sj = -0.5 * p->chord + (j + 0.5) * G->lb;
        G->bx[j] = G->xw + sj * G->tx;
        G->bz[j] = G->zw + sj * G->tz;
    }
    double ds = p->shed_offset * p->chord;
    G->lev_x = G->cx[0] - ds * G->tx;
    G->lev_z = G->cz[0] - ds * G->tz;
    G->tev_x = G->cx[G->n_c - 1] + ds * G->tx;
    G->tev_z = G->cz[G->n_c - 1] + ds * G->tz;
}

/* Packs [xw, zw, tx, tz, nx, nz, vx, vz, omega, cx(n_c), cz(n_c), bx(n_b), bz(n_b),
 *        lev_x, lev_z, tev_x, tev_z]. */
void ora_plate_geometry(const ora_params *p, const double *xg, double *out)
{
    ora_geom G;
    plate_geometry(p, xg, &G);
    int k = 0;
    out[k++] = G.xw; out[k++] = G.zw; out[k++] = G.tx; out[k++] = G.tz;
    out[k++] = G.nx; out[k++] = G.nz; out[k++] = G.vx; out[k++] = G.vz; out[k++] = G.omega;
    for (int i = 0; i < G.n_c; ++i) out[k++] = G.cx[i];
    for (int i = 0; i < G.n_c; ++i) out[k++] = G.cz[i];
    for (int j = 0; j < G.n_b; ++j) out[k++] = G.bx[j];
    for (int j = 0; j < G.n_b; ++j) out[k++] = G.bz[j];
    out[k++] = G.lev_x; out[k++] = G.lev_z; out[k++] = G.tev_x; out[k++] = G.tev_z;
}

/* Relative velocity at a surface point (Eq. 12, with the reading stated above). */
static void relative_velocity(const ora_params *p, const ora_geom *G, int n, const double *x,
                              const double *z, const double *g, double sx, double sz,
                              double *u, double *w)
{
    double wu, ww;
    induced(p->wake_kernel, p->r_core, n, x, z, g, sx, sz, -1, &wu, &ww);
    double rx = sx - G->xw, rz = sz - G->zw;        /* r_s - r_g */
    double ex = -rz, ez = rx;                       /* e_z x (r_s - r_g) */
    *u = wu + p->u_inf_x - G->vx - G->omega * ex;
    *w = ww + p->u_inf_z - G->vz - G->omega * ez;
}

/* ------------------------------------------------------------------ pressure and loads */

/* Pressure jump of Eq. 13 on each panel and the wing load and moment of Eqs. 14-15, from the
 * surface circulations gs (n_b bound, then Gamma_LEV, Gamma_TEV; 0 for an edge that shed
 * nothing), the previous step's bound circulations gb_prev (has_prev = 0 on the first step)
 * and the relative velocity (vbx, vbz) at the bound points (Eq. 12). fm = (F_w,x, F_w,z, M_w). */
static void plate_loads(const ora_params *p, const ora_geom *G, const double *gs,
                        const double *gb_prev, int has_prev, const double *vbx, const double *vbz,
                        double *fm)
{
    int nb = p->n_b;
    double dt = p->dt;
    double fwx = 0.0, fwz = 0.0, mw = 0.0;
    double cum = 0.0, cum_prev = 0.0;
    for (int i = 0; i < nb; ++i) {
        cum += gs[i];
        cum_prev += gb_prev[i];
        double tang = (gs[i] / G->lb) * (vbx[i] * G->tx + vbz[i] * G->tz);
        double dsum = has_prev ? (cum - cum_prev) / dt : 0.0;
        double dlev = has_prev ? gs[nb] / dt : 0.0;     /* the new LEV's circulation over dt */
        double dp = p->rho * (tang + dsum + dlev);
        double fx = G->lb * p->span * dp * G->nx, fz = G->lb * p->span * dp * G->nz;
        fwx += fx;
        fwz += fz;
        double ax = G->bx[i] - G->xw, az = G->bz[i] - G->zw;
        mw += ax * fz - az * fx;
    }
    fm[0] = fwx; fm[1] = fwz; fm[2] = mw;
}

/* The loads above for glider state xg, with vt the relative velocities at the plate points as
 * ora_step writes them (N_b + 1 collocation points, then N_b bound points, as (u, w) pairs). */
void ora_plate_loads(const ora_params *p, const double *xg, const double *gs,
                     const double *gb_prev, int has_prev, const double *vt, double *fm)
{
    ora_geom G;
    plate_geometry(p, xg, &G);
    int nb = p->n_b, nc = p->n_b + 1;
    double vbx[ORA_MAXB], vbz[ORA_MAXB];
    for (int j = 0; j < nb; ++j) { vbx[j] = vt[2 * (nc + j)]; vbz[j] = vt[2 * (nc + j) + 1]; }
    plate_loads(p, &G, gs, gb_prev, has_prev, vbx, vbz, fm);
}

/* ------------------------------------------------------------------ dense LU solve */

/* Solves A y = b in place (b <- y) by Gaussian elimination with partial pivoting. A is
 * row-major n x n and is overwritten by its factors. */
static int lu_solve(int n, double *A, double *b)
{
    for (int k = 0; k < n; ++k) {
        int piv = k;
        double best = fabs(A[k * n + k]);
        for (int i = k + 1; i < n; ++i)
            if (fabs(A[i * n + k]) > best) { best = fabs(A[i * n + k]); piv = i; }
        if (best == 0.0) return ORA_ERR_SINGULAR;
        if (piv != k) {
            for (int j = 0; j < n; ++j) {
                double t = A[k * n + j]; A[k * n + j] = A[piv * n + j]; A[piv * n + j] = t;
            }
            double t = b[k]; b[k] = b[piv]; b[piv] = t;
        }
        for (int i = k + 1; i < n; ++i) {
            double m = A[i * n + k] / A[k * n + k];
            A[i * n + k] = m;
            for (int j = k + 1; j < n; ++j) A[i * n + j] -= m * A[k * n + j];
            b[i] -= m * b[k];
        }
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = b[i];
        for (int j = i + 1; j < n; ++j) s -= A[i * n + j] * b[j];
        b[i] = s / A[i * n + i];
    }
    return ORA_OK;
}

/* ------------------------------------------------------------------ glider (§III-B) */

/* Time derivative of the glider state x_g = [x, z, th, phi, xd, zd, thd] under the wing load
 * (fwx, fwz, mw) and elevator rate u (Eqs. 18-22). */
static void glider_rhs(const ora_params *p, const double *xg, double fwx, double fwz, double mw,
                       double u, double *f)
{
    double th = xg[2], ph = xg[3], xd = xg[4], zd = xg[5], thd = xg[6];
    double ct = cos(th), st = sin(th), cp = cos(th + ph), sp = sin(th + ph);
    /* elevator velocity, Eq. 18 */
    double xed = xd + p->l * thd * st + p->l_e * (thd + u) * sp;
    double zed = zd - p->l * thd * ct - p->l_e * (thd + u) * cp;
    /* flat-plate elevator force, Eqs. 19-20 */
    double alpha_e = th + ph - atan2(zed, xed);
    double cn = 2.0 * sin(alpha_e);
    double q = 0.5 * p->rho * (xed * xed + zed * zed) * p->s_e * cn;
    double fex = q * (-sp), fez = q * cp;
    /* world-frame arms of the wing centre and the elevator from the centre of gravity */
    double awx = -p->l_w * ct, awz = -p->l_w * st;
    double aex = -p->l * ct - p->l_e * cp, aez = -p->l * st - p->l_e * sp;
    double torque = (awx * fwz - awz * fwx) + (aex * fez - aez * fex) + mw;
    f[0] = xd;
    f[1] = zd;
    f[2] = thd;
    f[3] = u;
    f[4] = (fwx + fex) / p->mass;
    f[5] = (fwz + fez) / p->mass - p->g;
    f[6] = torque / p->inertia;
}

void ora_glider_rhs(const ora_params *p, const double *xg, double fwx, double fwz, double mw,
                    double u, double *f)
{
    glider_rhs(p, xg, fwx, fwz, mw, u, f);
}

/* Terminal cost of Eq. 24. */
static double terminal_cost(const ora_params *p, const double *xg)
{
    double J = 0.0;
    for (int k = 0; k < 7; ++k) {
        double d = xg[k] - p->x_d[k];
        J += d * p->q[k] * d;
    }
    return J;
}

double ora_terminal_cost(const ora_params *p, const double *xg) { return terminal_cost(p, xg); }

/* ------------------------------------------------------------------ one VPM step */

/*
 * Advances the coupled state by one step of dt under elevator rate u.
 *   n, x, z, g     : wake particles (in/out; capacity entries allocated)
 *   xg             : glider state (7, in/out)
 *   gb_prev        : bound circulations of the previous step (n_b, in/out)
 *   glev_prev      : LEV circulation of the previous step (in/out; kept with the state, not
 *                    needed by Eq. 13 under the reading above)
 *   has_prev       : 0 on the first step (time derivatives are zero), set to 1
 * Optional outputs (NULL to skip):
 *   out_gs         : Gamma_S = [Gamma_b(n_b), Gamma_LEV, Gamma_TEV]
 *   out_fm         : [F_w,x, F_w,z, M_w]
 *   out_vel        : (u, w) of every particle of the enlarged wake, 2 * (n + shed)
 *   out_vt         : relative velocities at the n_c collocation points then the n_b bound
 *                    points, 2 * (n_c + n_b)
 *   out_alpha      : angle of attack used by the separation gate
 *   out_shed       : number of vortices shed this step (0, 1 or 2)
 */
/* Orientation of c relative to the directed line a -> b (twice the signed triangle area). */
static double orient(double ax, double az, double bx, double bz, double cx, double cz)
{
    return (bx - ax) * (cz - az) - (bz - az) * (cx - ax);
}

/* Whether segments p0-p1 and a-b cross (each segment's ends strictly on opposite sides of the
 * other's line; touching and collinear overlap do not count). */
static int segments_cross(double p0x, double p0z, double p1x, double p1z, double ax, double az,
                          double bx, double bz)
{
    double o1 = orient(ax, az, bx, bz, p0x, p0z), o2 = orient(ax, az, bx, bz, p1x, p1z);
    double o3 = orient(p0x, p0z, p1x, p1z, ax, az), o4 = orient(p0x, p0z, p1x, p1z, bx, bz);
    return ((o1 > 0.0 && o2 < 0.0) || (o1 < 0.0 && o2 > 0.0)) &&
           ((o3 > 0.0 && o4 < 0.0) || (o3 < 0.0 && o4 > 0.0));
}

static int step_impl(const ora_params *p, int capacity, int *n_io, double *x, double *z, double *g,
                     double *xg, double *gb_prev, double *glev_prev, int *has_prev, double u,
                     double *out_gs, double *out_fm, double *out_vel, double *out_vt,
                     double *out_alpha, int *out_shed, int *n_dist);

int ora_step(const ora_params *p, int capacity, int *n_io, double *x, double *z, double *g,
             double *xg, double *gb_prev, double *glev_prev, int *has_prev, double u,
             double *out_gs, double *out_fm, double *out_vel, double *out_vt, double *out_alpha,
             int *out_shed)
{
    int nd = 0;
    return step_impl(p, capacity, n_io, x, z, g, xg, gb_prev, glev_prev, has_prev, u, out_gs,
                     out_fm, out_vel, out_vt, out_alpha, out_shed, &nd);
}

/*
 * ora_step with a disturbance pair (§V): when *n_dist is 2 the first two particles are the
 * pair of opposite vortices standing for the vortex ring. They are convected with the wake
 * and are left out of merging. After the glider update, the pair is removed (*n_dist becomes
 * 0) once the segment joining it crosses the chord line offset by 2 % of the chord against
 * the normal, with the plate in its updated position.
 */
int ora_step_dist(const ora_params *p, int capacity, int *n_io, double *x, double *z, double *g,
                  double *xg, double *gb_prev, double *glev_prev, int *has_prev, double u,
                  double *out_gs, double *out_fm, double *out_vel, double *out_vt,
                  double *out_alpha, int *out_shed, int *n_dist)
{
    return step_impl(p, capacity, n_io, x, z, g, xg, gb_prev, glev_prev, has_prev, u, out_gs,
                     out_fm, out_vel, out_vt, out_alpha, out_shed, n_dist);
}

static int step_impl(const ora_params *p, int capacity, int *n_io, double *x, double *z, double *g,
                     double *xg, double *gb_prev, double *glev_prev, int *has_prev, double u,
                     double *out_gs, double *out_fm, double *out_vel, double *out_vt,
                     double *out_alpha, int *out_shed, int *n_dist)
{
    int n = *n_io;
    int nb = p->n_b, nc = p->n_b + 1;
    if (nb < 2 || nb > ORA_MAXB) return ORA_ERR_INVALID;
    ora_geom G;
    plate_geometry(p, xg, &G);

    /* separation gate: angle of attack of the wing relative to the surrounding air.
     * shed_gate 0: LEV and TEV shed every step; 1: neither is shed while |alpha| <= alpha_crit;
     * 2: the TEV is shed every step and the LEV only while |alpha| > alpha_crit. */
    double rel_x = G.vx - p->u_inf_x, rel_z = G.vz - p->u_inf_z;
    double alpha = xg[2] - atan2(rel_z, rel_x);
    alpha = atan2(sin(alpha), cos(alpha));
    if (out_alpha) *out_alpha = alpha;
    int open = fabs(alpha) > p->alpha_crit;
    int shed_lev = (p->shed_gate == 0) || open;
    int shed_tev = (p->shed_gate != 1) || open;
    if (out_shed) *out_shed = shed_lev + shed_tev;
    if (n + shed_lev + shed_tev > capacity) return ORA_ERR_CAPACITY;

    /* relative velocity at the collocation and bound points from the wake W (Eq. 12) */
    double vcx[ORA_MAXB + 1], vcz[ORA_MAXB + 1], vbx[ORA_MAXB], vbz[ORA_MAXB];
    for (int i = 0; i < nc; ++i)
        relative_velocity(p, &G, n, x, z, g, G.cx[i], G.cz[i], &vcx[i], &vcz[i]);
    for (int j = 0; j < nb; ++j)
        relative_velocity(p, &G, n, x, z, g, G.bx[j], G.bz[j], &vbx[j], &vbz[j]);
    if (out_vt) {
        for (int i = 0; i < nc; ++i) { out_vt[2 * i] = vcx[i]; out_vt[2 * i + 1] = vcz[i]; }
        for (int j = 0; j < nb; ++j) {
            out_vt[2 * (nc + j)] = vbx[j]; out_vt[2 * (nc + j) + 1] = vbz[j];
        }
    }

    /* Kelvin bookkeeping: total wake circulation (Eq. 7) */
    double gw = 0.0;
    for (int v = 0; v < n; ++v) gw += g[v];

    /* surface circulation system (Eqs. 8-11), assembled and solved by LU every step.
     * Unknowns: the bound circulations, then Gamma_LEV and Gamma_TEV when they are shed.
     * Rows: the no-through-flow condition (Eq. 6) at each collocation point (the LE row is
     * dropped when no LEV is shed, the TE row when no TEV is shed), then Kelvin's row. */
    int m = nb + shed_lev + shed_tev;
    double A[(ORA_MAXB + 2) * (ORA_MAXB + 2)], b[ORA_MAXB + 2];
    int r = 0;
    for (int i = 0; i < nc; ++i) {
        if (i == 0 && !shed_lev) continue;
        if (i == nc - 1 && !shed_tev) continue;
        int col = 0;
        for (int j = 0; j < nb; ++j) {
            double kx, kz;
            kernel_eval(ORA_SINGULAR, 0.0, G.cx[i] - G.bx[j], G.cz[i] - G.bz[j], &kx, &kz);
            A[r * m + col++] = kx * G.nx + kz * G.nz;
        }
        if (shed_lev) {
            double kx, kz;
            kernel_eval(p->wake_kernel, p->r_core, G.cx[i] - G.lev_x, G.cz[i] - G.lev_z, &kx, &kz);
            A[r * m + col++] = kx * G.nx + kz * G.nz;
        }
        if (shed_tev) {
            double kx, kz;
            kernel_eval(p->wake_kernel, p->r_core, G.cx[i] - G.tev_x, G.cz[i] - G.tev_z, &kx, &kz);
            A[r * m + col++] = kx * G.nx + kz * G.nz;
        }
        b[r] = -(vcx[i] * G.nx + vcz[i] * G.nz);
        ++r;
    }
    for (int j = 0; j < m; ++j) A[r * m + j] = 1.0;
    b[r] = -gw;
    int rc = lu_solve(m, A, b);
    if (rc != ORA_OK) return rc;
    double gs[ORA_MAXB + 2];
    for (int j = 0; j < nb; ++j) gs[j] = b[j];
    gs[nb] = shed_lev ? b[nb] : 0.0;
    gs[nb + 1] = shed_tev ? b[nb + shed_lev] : 0.0;
    if (out_gs) for (int j = 0; j < nb + 2; ++j) out_gs[j] = gs[j];

    /* unsteady Bernoulli pressure jump (Eq. 13) and wing loads (Eqs. 14-15) */
    double dt = p->dt;
    double fm[3];
    plate_loads(p, &G, gs, gb_prev, *has_prev, vbx, vbz, fm);
    double fwx = fm[0], fwz = fm[1], mw = fm[2];
    if (out_fm) { out_fm[0] = fwx; out_fm[1] = fwz; out_fm[2] = mw; }

    /* W <- W u E (LEV first, then TEV) */
    if (shed_lev) { x[n] = G.lev_x; z[n] = G.lev_z; g[n] = gs[nb]; ++n; }
    if (shed_tev) { x[n] = G.tev_x; z[n] = G.tev_z; g[n] = gs[nb + 1]; ++n; }

    /* convection velocities of the enlarged wake (Eq. 16) plus the free stream */
    double *uu = malloc(sizeof(double) * (n > 0 ? n : 1));
    double *ww = malloc(sizeof(double) * (n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) {
        double su, sw;
        induced(p->wake_kernel, p->r_core, n, x, z, g, x[i], z[i], i, &su, &sw);
        double bu, bw;
        induced(ORA_SINGULAR, 0.0, nb, G.bx, G.bz, gs, x[i], z[i], -1, &bu, &bw);
        uu[i] = su + bu + p->u_inf_x;
        ww[i] = sw + bw + p->u_inf_z;
    }
    if (out_vel) for (int i = 0; i < n; ++i) { out_vel[2 * i] = uu[i]; out_vel[2 * i + 1] = ww[i]; }

    /* explicit Euler advection and circulation decay (Eq. 17, exact decay over dt) */
    double decay = exp(-p->gamma_decay * dt);
    for (int i = 0; i < n; ++i) {
        x[i] += dt * uu[i];
        z[i] += dt * ww[i];
        g[i] *= decay;
    }
    free(uu); free(ww);

    /* glider explicit Euler update under the loads of this step */
    if (!p->fixed_plate) {
        double f[7];
        glider_rhs(p, xg, fwx, fwz, mw, u, f);
        for (int k = 0; k < 7; ++k) xg[k] += dt * f[k];
    }

    /* disturbance termination: the pair's segment against the offset chord line */
    if (*n_dist == 2 && n >= 2) {
        ora_geom G2;
        plate_geometry(p, xg, &G2);
        double off = 0.02 * p->chord;
        double ax = G2.cx[0] - off * G2.nx, az = G2.cz[0] - off * G2.nz;
        double bx = G2.cx[nc - 1] - off * G2.nx, bz = G2.cz[nc - 1] - off * G2.nz;
        if (segments_cross(x[0], z[0], x[1], z[1], ax, az, bx, bz)) {
            for (int v = 0; v + 2 < n; ++v) { x[v] = x[v + 2]; z[v] = z[v + 2]; g[v] = g[v + 2]; }
            n -= 2;
            *n_dist = 0;
        }
    }

    /* merge the two oldest wake particles (after the disturbance pair, which is left alone)
     * while the wake is over its limit */
    if (p->n_wake_max > 0) {
        int d = *n_dist;
        while (n - d > p->n_wake_max && n - d >= 2) {
            x[d] = 0.5 * (x[d] + x[d + 1]);
            z[d] = 0.5 * (z[d] + z[d + 1]);
            g[d] = g[d] + g[d + 1];
            for (int v = d + 1; v + 1 < n; ++v) { x[v] = x[v + 1]; z[v] = z[v + 1]; g[v] = g[v + 1]; }
            n -= 1;
        }
    }

    for (int j = 0; j < nb; ++j) gb_prev[j] = gs[j];
    *glev_prev = gs[nb];
    *has_prev = 1;
    *n_io = n;
    return ORA_OK;
}

/*
 * One rollout of H steps from a root state, which is copied and not modified. controls[H]
 * are the elevator rates. Outputs: final glider state, terminal cost (Eq. 24), optional
 * trajectory traj[H][7] (glider state after each step) and optional final wake.
 */
int ora_rollout(const ora_params *p, int capacity, int n0, const double *x0, const double *z0,
                const double *g0, const double *xg0, const double *gb_prev0, double glev_prev0,
                int has_prev0, int H, const double *controls, double *out_xg, double *out_cost,
                double *out_traj, int *out_n, double *out_x, double *out_z, double *out_g,
                int n_dist0)
{
    int nd = n_dist0;
    double *x = malloc(sizeof(double) * capacity);
    double *z = malloc(sizeof(double) * capacity);
    double *g = malloc(sizeof(double) * capacity);
    double xg[7], gbp[ORA_MAXB], glp = glev_prev0;
    int n = n0, hp = has_prev0, rc = ORA_OK;
    memcpy(x, x0, sizeof(double) * n0);
    memcpy(z, z0, sizeof(double) * n0);
    memcpy(g, g0, sizeof(double) * n0);
    memcpy(xg, xg0, sizeof(xg));
    for (int j = 0; j < p->n_b; ++j) gbp[j] = gb_prev0 ? gb_prev0[j] : 0.0;
    for (int k = 0; k < H && rc == ORA_OK; ++k) {
        rc = step_impl(p, capacity, &n, x, z, g, xg, gbp, &glp, &hp, controls[k], NULL, NULL,
                       NULL, NULL, NULL, NULL, &nd);
        if (out_traj) memcpy(out_traj + 7 * k, xg, sizeof(xg));
    }
    if (out_xg) memcpy(out_xg, xg, sizeof(xg));
    if (out_cost) *out_cost = terminal_cost(p, xg);
    if (out_n) *out_n = n;
    if (out_x) memcpy(out_x, x, sizeof(double) * n);
    if (out_z) memcpy(out_z, z, sizeof(double) * n);
    if (out_g) memcpy(out_g, g, sizeof(double) * n);
    free(x); free(z); free(g);
    return rc;
}

/* ------------------------------------------------------------------ MPPI (§IV-A, Eq. 25) */

/* w_i = eta exp(-(J_i - J_min)/lambda), eta = 1 / sum_i exp(-(J_i - J_min)/lambda), J_min and
 * the sum over the finite costs. A cost that is not finite (a rollout that diverged) takes the
 * limit of Eq. 25 as J_i -> +inf: weight 0. With no finite cost every weight is NaN. */
void ora_mppi_weights(int K, const double *J, double lambda, double *w)
{
    double jmin = INFINITY;
    int finite = 0;
    for (int i = 0; i < K; ++i)
        if (isfinite(J[i])) { finite = 1; if (J[i] < jmin) jmin = J[i]; }
    if (!finite) { for (int i = 0; i < K; ++i) w[i] = NAN; return; }
    double s = 0.0;
    for (int i = 0; i < K; ++i) { w[i] = isfinite(J[i]) ? exp(-(J[i] - jmin) / lambda) : 0.0; s += w[i]; }
    double eta = 1.0 / s;
    for (int i = 0; i < K; ++i) w[i] *= eta;
}

/* xi_hat = sum_i w_i xi_i over K sequences of H controls (xi row-major K x H). */
void ora_mppi_update(int K, int H, const double *w, const double *xi, double *mu)
{
    for (int k = 0; k < H; ++k) {
        double s = 0.0;
        for (int i = 0; i < K; ++i) s += w[i] * xi[(size_t)i * H + k];
        mu[k] = s;
    }
}

/*
 * chcpic_oracle.c -- plain, slow, FP64 CPU oracle for one time step of the
 * charge-conserving particle-in-cell (ChCPIC) scheme with the alternating-order
 * form factor of order l_a = 1 1/2 or 2 1/2 (I. V. Sokolov, "Alternating-Order
 * Interpolation in a Charge-Conserving Scheme for Particle-In-Cell
 * Simulations", arXiv:1101.0809).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness reference that the
 * CUDA library is checked against.  Only the test suite, the package smoke
 * check and the benchmark's CPU-baseline leg may load it.  It shares no code,
 * header, table or constant with the CUDA path and never calls it; the CUDA
 * path never calls it either.
 *
 * Everything is double precision, single threaded, one particle at a time in
 * storage order, in the order of the paper's Appendix.  Nothing is blocked,
 * fused or reordered.
 *
 * Conventions (Sec. 2 of the paper):
 *   - Normalized coordinates x~ = x/dx, t~ = t/dt (Eq. coorddimless); a
 *     particle position is an absolute real number per axis, kept in [0, N).
 *     c_a = c*dt/d_a are the Courant numbers.
 *   - Yee staggering (Sec. 2).  Array element [i,j,k] holds
 *         Ex at (i, j+1/2, k+1/2)   Ey at (i+1/2, j, k+1/2)   Ez at (i+1/2, j+1/2, k)
 *         Bx at (i+1/2, j, k)       By at (i, j+1/2, k)       Bz at (i, j, k+1/2)
 *     J is placed like E; rho at (i+1/2, j+1/2, k+1/2).  Arrays are x-fastest:
 *     linear index = (k*ny + j)*nx + i, all indices periodic.
 *   - 2D3V runs (dims == 2) have an ignorable z: nz == 1, every interpolation
 *     weight loses its z factor (its sum over k is 1, Eq. one), and the current
 *     is the 3D current of Eq. current summed over the ignorable index k.
 *   - Gaussian units (Eqs. 1-4).
 *
 * Parity pins for every function here live in tests/test_oracle_pins.py.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int dims;              /* 2 or 3 */
    int nx, ny, nz;        /* cells per axis (nz == 1 when dims == 2) */
    double dx, dy, dz;     /* cell sizes */
    double dt, c;          /* time step, speed of light */
    int order2;            /* 3 (l_a = 1 1/2; also 0), 5 (l_a = 2 1/2), or 4: the uniform-order l = 2
                              comparison scheme of Eq. wrong1 */
} orc_grid;

typedef struct {
    double q, m, weight;   /* physical charge and mass; macro-particle weight */
    long long n;           /* number of macro-particles */
    double *x[3];          /* normalized absolute positions, each in [0, N_a) */
    double *w[3];          /* momentum-to-mass ratio w = gamma*v */
} orc_species;

typedef struct {
    double kinetic;        /* sum m_p c (sqrt(w^2+c^2) - c), w at n-1/2 */
    double field_E;        /* V/(8 pi) sum E^2 at time n */
    double field_B;        /* V/(8 pi) sum B^2 at time n */
    double half_step_corr; /* sum (q_p dt/2) u^{n-1/2} . E(x^n) */
    double total;          /* sum of the four terms above */
    double momentum[3];    /* sum m_p w */
    double charge;         /* V * sum rho over cells (particles + background) */
} orc_diag;

static const double ORC_PI = 3.14159265358979323846;

static long long wrap_index(long long i, long long n)
{
    long long m = i % n;
    return m < 0 ? m + n : m;
}

static long long cell_index(const orc_grid *g, long long i, long long j, long long k)
{
    return (wrap_index(k, g->nz) * g->ny + wrap_index(j, g->ny)) * g->nx + wrap_index(i, g->nx);
}

static double cell_volume(const orc_grid *g)
{
    return g->dims == 2 ? g->dx * g->dy : g->dx * g->dy * g->dz;
}

/* ---------------------------------------------------------------------------
 * Alternating-order form factor (Sec. 4.5, closed-form values).  The weight of
 * a grid point is f^(l) at integer points and dF = f^(l+1) at half-integer
 * points (the cell integrals of f^(l), Eq. intff); l_a = l + 1/2.
 *
 * l_a = 1 1/2: with i = int(x_p) and d = x_p - i,
 *   f at the integer points i, i+1:                      (1-d, d)
 *   dF at the half-integers i-1/2, i+1/2, i+3/2:         ((1-d)^2/2, 3/4 - (1/2-d)^2, d^2/2)
 * l_a = 2 1/2: with i = int(x_p + 1/2) and d = x_p + 1/2 - i,
 *   f at the integer points i-1, i, i+1:                 ((1-d)^2/2, 3/4 - (1/2-d)^2, d^2/2)
 *   dF at the half-integers i-3/2, ..., i+3/2:
 *        ((1-d)^3/6, (2-d)^3/6 - 2(1-d)^3/3, (1+d)^3/6 - 2d^3/3, d^3/6)
 * "int" is read as floor on the wrapped, non-negative position.  The
 * half-integer point c+1/2 is the centre of cell c.
 *
 * The comparison scheme of Eq. wrong1 (Sec. 5, the "conventional" l = 2
 * interpolation) keeps the l_a = 1 1/2 cell integrals dF at half-integer points
 * and replaces the point values at an integer point i by the mean of the two
 * neighbouring cell integrals, (dF_{i-1/2} + dF_{i+1/2})/2: the cell-centred
 * weight applied to the field averaged over the two faces of the cell.  With
 * dF nonzero on the cells i0-1 .. i0+1 this gives four integer points
 * i0-1 .. i0+2.  The deposit and rho are those of l_a = 1 1/2.
 * ------------------------------------------------------------------------- */
void orc_form_factor(double xp, long long *i, double f[2], double dF[3])
{
    double fl = floor(xp);
    double d = xp - fl;
    *i = (long long)fl;
    f[0] = 1.0 - d;
    f[1] = d;
    dF[0] = 0.5 * (1.0 - d) * (1.0 - d);
    dF[1] = 0.75 - (0.5 - d) * (0.5 - d);
    dF[2] = 0.5 * d * d;
}

void orc_form_factor5(double xp, long long *i, double f[3], double dF[4])
{
    double fl = floor(xp + 0.5);
    double d = xp + 0.5 - fl;
    double e = 1.0 - d;
    *i = (long long)fl;
    f[0] = 0.5 * e * e;
    f[1] = 0.75 - (0.5 - d) * (0.5 - d);
    f[2] = 0.5 * d * d;
    dF[0] = e * e * e / 6.0;
    dF[1] = (2.0 - d) * (2.0 - d) * (2.0 - d) / 6.0 - 2.0 * e * e * e / 3.0;
    dF[2] = (1.0 + d) * (1.0 + d) * (1.0 + d) / 6.0 - 2.0 * d * d * d / 3.0;
    dF[3] = d * d * d / 6.0;
}

static int grid_order2(const orc_grid *g) { return g->order2 == 5 || g->order2 == 4 ? g->order2 : 3; }

/* Weights of one axis: nf point values f at the integer points ib+fo+a
 * (a = 0..nf-1) and nS cell integrals dF over the cells ib+so+b (b = 0..nS-1). */
typedef struct {
    long long ib;
    int nf, fo, nS, so;
    double f[4];
    double dF[4];
} orc_axis_w;

static void axis_weights(int order2, double xp, orc_axis_w *w)
{
    if (order2 == 5) {
        orc_form_factor5(xp, &w->ib, w->f, w->dF);
        w->nf = 3; w->fo = -1; w->nS = 4; w->so = -2;
    } else if (order2 == 4) {   /* Eq. wrong1 */
        double f1[2];
        orc_form_factor(xp, &w->ib, f1, w->dF);
        w->nS = 3; w->so = -1;
        w->nf = 4; w->fo = -1;
        w->f[0] = 0.5 * w->dF[0];
        w->f[1] = 0.5 * (w->dF[0] + w->dF[1]);
        w->f[2] = 0.5 * (w->dF[1] + w->dF[2]);
        w->f[3] = 0.5 * w->dF[2];
    } else {
        orc_form_factor(xp, &w->ib, w->f, w->dF);
        w->nf = 2; w->fo = 0; w->nS = 3; w->so = -1;
    }
}

/* Per-axis weights of one particle.  In 2D the z axis is degenerate: one
 * point k = 0 with weight 1 for both kinds of point, which drops the z factor
 * from every product below. */
typedef struct {
    orc_axis_w ax[3];
} orc_weights;

static void particle_weights(const orc_grid *g, const double xp[3], orc_weights *wt)
{
    for (int a = 0; a < 3; ++a) {
        orc_axis_w *w = &wt->ax[a];
        if (a == 2 && g->dims == 2) {
            w->ib = 0;
            w->nf = 1; w->fo = 0; w->f[0] = 1.0;
            w->nS = 1; w->so = 0; w->dF[0] = 1.0;
            continue;
        }
        axis_weights(grid_order2(g), xp[a], w);
    }
}

/* Interpolation sum of one staggered grid function at the particle: along axis
 * a over the integer points with f when ipt[a] is set, else over the cells
 * with dF.  F[i,j,k] sits at i (integer) or i+1/2 (cell centre) per axis. */
static double interp_point(const orc_grid *g, const orc_weights *wt, const int ipt[3], const double *F)
{
    const orc_axis_w *X = &wt->ax[0], *Y = &wt->ax[1], *Z = &wt->ax[2];
    const int nx = ipt[0] ? X->nf : X->nS, ny = ipt[1] ? Y->nf : Y->nS, nz = ipt[2] ? Z->nf : Z->nS;
    const int ox = ipt[0] ? X->fo : X->so, oy = ipt[1] ? Y->fo : Y->so, oz = ipt[2] ? Z->fo : Z->so;
    const double *wx = ipt[0] ? X->f : X->dF, *wy = ipt[1] ? Y->f : Y->dF, *wz = ipt[2] ? Z->f : Z->dF;
    double acc = 0.0;
    for (int c = 0; c < nz; ++c)
        for (int b = 0; b < ny; ++b)
            for (int a = 0; a < nx; ++a)
                acc += wx[a] * wy[b] * wz[c] * F[cell_index(g, X->ib + ox + a, Y->ib + oy + b, Z->ib + oz + c)];
    return acc;
}

/* ---------------------------------------------------------------------------
 * Field gather (Sec. 2 interpolation sums, weights alpha of Eq. alphax and
 * beta of Eq. betax).  Along its own axis an E component takes the lower-order
 * point values f at integer points; along the two other axes it takes the cell
 * integrals dF at half-integer points.  A B component is the other way round.
 *   E^(x) at (i, j+1/2, k+1/2): alpha^(x) = f_i(x) dF_{j+1/2}(y) dF_{k+1/2}(z), cyclically;
 *   B^(x) at (i+1/2, j, k):     beta^(x)  = dF_{i+1/2}(x) f_j(y) f_k(z), cyclically.
 * In 2D the z factor is the single weight 1 for both kinds.
 * ------------------------------------------------------------------------- */
void orc_gather(const orc_grid *g, const double *const E[3], const double *const B[3],
                const double xp[3], double Ep[3], double Bp[3])
{
    orc_weights wt;
    particle_weights(g, xp, &wt);
    for (int a = 0; a < 3; ++a) {
        int ie[3] = { 0, 0, 0 }, ib[3] = { 1, 1, 1 };
        ie[a] = 1;   /* E^(a): integer points along a */
        ib[a] = 0;   /* B^(a): cells along a */
        Ep[a] = interp_point(g, &wt, ie, E[a]);
        Bp[a] = interp_point(g, &wt, ib, B[a]);
    }
}

/* ---------------------------------------------------------------------------
 * Relativistic momentum push (Appendix, step 2; Eq. 1), with q/m and dt:
 *   e = q dt/(2m) E;  w~ = w + e;  b = q dt/(2 m sqrt(w~^2 + c^2)) B;
 *   w_n = w~ + w~ x b;  w' = w~ + e + 2 (w_n x b)/(1 + b^2).
 * ------------------------------------------------------------------------- */
static void cross(const double a[3], const double b[3], double r[3])
{
    r[0] = a[1] * b[2] - a[2] * b[1];
    r[1] = a[2] * b[0] - a[0] * b[2];
    r[2] = a[0] * b[1] - a[1] * b[0];
}

void orc_boris(double w[3], const double Ep[3], const double Bp[3], double qm, double dt, double c)
{
    double e[3], wt[3], b[3], wn[3], t[3];
    for (int a = 0; a < 3; ++a) e[a] = 0.5 * qm * dt * Ep[a];
    for (int a = 0; a < 3; ++a) wt[a] = w[a] + e[a];
    double gam = sqrt(wt[0] * wt[0] + wt[1] * wt[1] + wt[2] * wt[2] + c * c);
    for (int a = 0; a < 3; ++a) b[a] = 0.5 * qm * dt * Bp[a] / gam;
    cross(wt, b, t);
    for (int a = 0; a < 3; ++a) wn[a] = wt[a] + t[a];
    double b2 = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
    cross(wn, b, t);
    for (int a = 0; a < 3; ++a) w[a] = wt[a] + e[a] + 2.0 * t[a] / (1.0 + b2);
}

/* Velocity and new position (Appendix, Eq. coordscheme):
 *   u/c = w / sqrt(w^2 + c^2);  x^{n+1} = x^n + (u/c) . diag(c_x, c_y, c_z).
 * The returned position is NOT wrapped into the box.  In 2D, x1[2] = x0[2]. */
void orc_move(const orc_grid *g, const double w[3], const double x0[3], double x1[3], double u[3])
{
    double gam = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2] + g->c * g->c);
    double cN[3] = { g->c * g->dt / g->dx, g->c * g->dt / g->dy, g->c * g->dt / g->dz };
    for (int a = 0; a < 3; ++a) u[a] = g->c * w[a] / gam;
    for (int a = 0; a < 3; ++a) x1[a] = x0[a] + (w[a] / gam) * cN[a];
    if (g->dims == 2) x1[2] = x0[2];
}

/* Periodic wrap of a position into [0, N) per axis. */
void orc_wrap(const orc_grid *g, double x[3])
{
    const int n[3] = { g->nx, g->ny, g->nz };
    for (int a = 0; a < g->dims; ++a) {
        double N = (double)n[a];
        while (x[a] < 0.0) {
            x[a] += N;
            if (x[a] >= N) x[a] = 0.0;   /* a tiny negative rounds up to N */
        }
        while (x[a] >= N) x[a] -= N;
    }
}

/* ---------------------------------------------------------------------------
 * Virtual-path current of one particle (Sec. 3.2, Eq. current; Appendix step 2d).
 * Per axis the cells touched by the old or the new cloud form the window
 * [lo, hi]; dF at x^n and at x^{n+1} are laid on it, dF(+-) = dF(x^{n+1}) +- dF(x^n),
 * and the partial sums D(i) = F_i(x^{n+1}) - F_i(x^n) = sum_{i' <= i} dF(-)_{i'-1/2}
 * give the face factor.  Then, for the x faces,
 *   xi^(x)_{i,j+1/2,k+1/2} = -(1/4)(dx/dt) D_x(i)
 *          [dF(+)_{j+1/2}(y) dF(+)_{k+1/2}(z) + (1/3) dF(-)_{j+1/2}(y) dF(-)_{k+1/2}(z)]
 * and cyclically for y, z; J += (q_p/V) xi (Eq. xi).
 * 2D (ignorable z): summing the 3D xi over k with sum_k dF(+)_z = 2,
 * sum_k dF(-)_z = 0 and sum_k D_z(k) = z^n - z^{n+1} (Eq. sumcurrent) gives
 *   xi^(x) = -(1/2)(dx/dt) D_x(i) dF(+)_{j+1/2}(y),
 *   xi^(y) = -(1/2)(dy/dt) D_y(j) dF(+)_{i+1/2}(x),
 *   xi^(z) = (1/4) u_z [dF(+)_x dF(+)_y + (1/3) dF(-)_x dF(-)_y].
 * x1 is the unwrapped new position; u is the velocity u^{n+1/2}.
 * Returns the largest |sum_window dF(-)| (exactly zero in exact arithmetic).
 * ------------------------------------------------------------------------- */
#define ORC_MAXWIN 16

typedef struct {
    long long lo;          /* first window cell */
    int len;               /* window cells lo .. lo+len-1 */
    double Pp[ORC_MAXWIN]; /* dF(+) per window cell */
    double Pm[ORC_MAXWIN]; /* dF(-) per window cell */
    double D[ORC_MAXWIN];  /* D at the face on the left of window cell s (s = 1..len-1) */
    double closure;        /* sum of dF(-) over the window */
} orc_axis_current;

static int axis_current(int order2, double x0, double x1, orc_axis_current *ac)
{
    orc_axis_w w0, w1;
    axis_weights(order2, x0, &w0);
    axis_weights(order2, x1, &w1);
    long long lo = (w0.ib < w1.ib ? w0.ib : w1.ib) + w0.so;
    long long hi = (w0.ib > w1.ib ? w0.ib : w1.ib) + w0.so + w0.nS - 1;
    int len = (int)(hi - lo + 1);
    if (len > ORC_MAXWIN) return -1;
    double old_w[ORC_MAXWIN], new_w[ORC_MAXWIN];
    for (int s = 0; s < len; ++s) { old_w[s] = 0.0; new_w[s] = 0.0; }
    for (int b = 0; b < w0.nS; ++b) {
        old_w[w0.ib + w0.so + b - lo] = w0.dF[b];
        new_w[w1.ib + w1.so + b - lo] = w1.dF[b];
    }
    ac->lo = lo;
    ac->len = len;
    for (int s = 0; s < len; ++s) {
        ac->Pp[s] = new_w[s] + old_w[s];
        ac->Pm[s] = new_w[s] - old_w[s];
    }
    /* D at face lo+s is the sum of dF(-) over the cells left of it */
    double run = 0.0;
    ac->D[0] = 0.0;
    for (int s = 1; s < len; ++s) {
        run += ac->Pm[s - 1];
        ac->D[s] = run;
    }
    ac->closure = run + ac->Pm[len - 1];
    return 0;
}

double orc_deposit(const orc_grid *g, const double x0[3], const double x1[3], const double u[3],
                   double qp, double *J[3])
{
    orc_axis_current ax[3];
    for (int a = 0; a < g->dims; ++a)
        if (axis_current(grid_order2(g), x0[a], x1[a], &ax[a]) != 0) return INFINITY;
    const double qV = qp / cell_volume(g);
    const double dtn = g->dt;
    double worst = 0.0;
    for (int a = 0; a < g->dims; ++a)
        if (fabs(ax[a].closure) > worst) worst = fabs(ax[a].closure);

    if (g->dims == 3) {
        /* x faces: face index i = lo_x + s (s = 1..len-1), cells j, k */
        for (int sk = 0; sk < ax[2].len; ++sk)
            for (int sj = 0; sj < ax[1].len; ++sj)
                for (int si = 1; si < ax[0].len; ++si) {
                    double xi = -0.25 * (g->dx / dtn) * ax[0].D[si] *
                                (ax[1].Pp[sj] * ax[2].Pp[sk] + ax[1].Pm[sj] * ax[2].Pm[sk] / 3.0);
                    J[0][cell_index(g, ax[0].lo + si, ax[1].lo + sj, ax[2].lo + sk)] += qV * xi;
                }
        /* y faces */
        for (int sk = 0; sk < ax[2].len; ++sk)
            for (int sj = 1; sj < ax[1].len; ++sj)
                for (int si = 0; si < ax[0].len; ++si) {
                    double xi = -0.25 * (g->dy / dtn) * ax[1].D[sj] *
                                (ax[0].Pp[si] * ax[2].Pp[sk] + ax[0].Pm[si] * ax[2].Pm[sk] / 3.0);
                    J[1][cell_index(g, ax[0].lo + si, ax[1].lo + sj, ax[2].lo + sk)] += qV * xi;
                }
        /* z faces */
        for (int sk = 1; sk < ax[2].len; ++sk)
            for (int sj = 0; sj < ax[1].len; ++sj)
                for (int si = 0; si < ax[0].len; ++si) {
                    double xi = -0.25 * (g->dz / dtn) * ax[2].D[sk] *
                                (ax[0].Pp[si] * ax[1].Pp[sj] + ax[0].Pm[si] * ax[1].Pm[sj] / 3.0);
                    J[2][cell_index(g, ax[0].lo + si, ax[1].lo + sj, ax[2].lo + sk)] += qV * xi;
                }
    } else {
        for (int sj = 0; sj < ax[1].len; ++sj)
            for (int si = 1; si < ax[0].len; ++si) {
                double xi = -0.5 * (g->dx / dtn) * ax[0].D[si] * ax[1].Pp[sj];
                J[0][cell_index(g, ax[0].lo + si, ax[1].lo + sj, 0)] += qV * xi;
            }
        for (int sj = 1; sj < ax[1].len; ++sj)
            for (int si = 0; si < ax[0].len; ++si) {
                double xi = -0.5 * (g->dy / dtn) * ax[1].D[sj] * ax[0].Pp[si];
                J[1][cell_index(g, ax[0].lo + si, ax[1].lo + sj, 0)] += qV * xi;
            }
        for (int sj = 0; sj < ax[1].len; ++sj)
            for (int si = 0; si < ax[0].len; ++si) {
                double xi = 0.25 * u[2] *
                            (ax[0].Pp[si] * ax[1].Pp[sj] + ax[0].Pm[si] * ax[1].Pm[sj] / 3.0);
                J[2][cell_index(g, ax[0].lo + si, ax[1].lo + sj, 0)] += qV * xi;
            }
    }
    return worst;
}

/* Charge density of one species (Eq. rho): rho_{i+1/2,...} += (q_p/V) dF_x dF_y dF_z
 * over the cells of the particle's dF window (3 or 4 per axis). */
void orc_rho(const orc_grid *g, long long n, const double *const x[3], double qp, double *rho)
{
    const double qV = qp / cell_volume(g);
    for (long long p = 0; p < n; ++p) {
        double xp[3] = { x[0][p], x[1][p], g->dims == 3 ? x[2][p] : 0.0 };
        orc_weights wt;
        particle_weights(g, xp, &wt);
        const orc_axis_w *X = &wt.ax[0], *Y = &wt.ax[1], *Z = &wt.ax[2];
        for (int c = 0; c < Z->nS; ++c)
            for (int b = 0; b < Y->nS; ++b)
                for (int a = 0; a < X->nS; ++a)
                    rho[cell_index(g, X->ib + X->so + a, Y->ib + Y->so + b, Z->ib + Z->so + c)] +=
                        qV * X->dF[a] * Y->dF[b] * Z->dF[c];
    }
}

/* ---------------------------------------------------------------------------
 * Yee field updates (Appendix, Eqs. updateB and escheme), completed cyclically.
 *   B half step:  B -= (1/2) c_h curl E, e.g.
 *     Bx[i,j,k] -= (c_y/2)(Ez[i,j,k]-Ez[i,j-1,k]) - (c_z/2)(Ey[i,j,k]-Ey[i,j,k-1])
 *   E full step:  E += -4 pi dt J + c_h curl B, e.g.
 *     Ex[i,j,k] += -4 pi dt Jx + c_y(Bz[i,j+1,k]-Bz[i,j,k]) - c_z(By[i,j,k+1]-By[i,j,k])
 * In 2D every z difference is zero.
 * ------------------------------------------------------------------------- */
void orc_yee_half_B(const orc_grid *g, const double *const E[3], double *B[3])
{
    const double cx = g->c * g->dt / g->dx, cy = g->c * g->dt / g->dy;
    const double cz = g->dims == 2 ? 0.0 : g->c * g->dt / g->dz;
    const long long N = (long long)g->nx * g->ny * g->nz;
    double *nb[3];
    for (int a = 0; a < 3; ++a) nb[a] = (double *)malloc(sizeof(double) * N);
    for (int k = 0; k < g->nz; ++k)
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i) {
                long long p = cell_index(g, i, j, k);
                nb[0][p] = B[0][p] - 0.5 * cy * (E[2][p] - E[2][cell_index(g, i, j - 1, k)])
                                   + 0.5 * cz * (E[1][p] - E[1][cell_index(g, i, j, k - 1)]);
                nb[1][p] = B[1][p] - 0.5 * cz * (E[0][p] - E[0][cell_index(g, i, j, k - 1)])
                                   + 0.5 * cx * (E[2][p] - E[2][cell_index(g, i - 1, j, k)]);
                nb[2][p] = B[2][p] - 0.5 * cx * (E[1][p] - E[1][cell_index(g, i - 1, j, k)])
                                   + 0.5 * cy * (E[0][p] - E[0][cell_index(g, i, j - 1, k)]);
            }
    for (int a = 0; a < 3; ++a) {
        memcpy(B[a], nb[a], sizeof(double) * N);
        free(nb[a]);
    }
}

void orc_yee_E(const orc_grid *g, const double *const B[3], const double *const J[3], double *E[3])
{
    const double cx = g->c * g->dt / g->dx, cy = g->c * g->dt / g->dy;
    const double cz = g->dims == 2 ? 0.0 : g->c * g->dt / g->dz;
    const double fpdt = 4.0 * ORC_PI * g->dt;
    for (int k = 0; k < g->nz; ++k)
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i) {
                long long p = cell_index(g, i, j, k);
                E[0][p] += -fpdt * J[0][p] + cy * (B[2][cell_index(g, i, j + 1, k)] - B[2][p])
                                           - cz * (B[1][cell_index(g, i, j, k + 1)] - B[1][p]);
                E[1][p] += -fpdt * J[1][p] + cz * (B[0][cell_index(g, i, j, k + 1)] - B[0][p])
                                           - cx * (B[2][cell_index(g, i + 1, j, k)] - B[2][p]);
                E[2][p] += -fpdt * J[2][p] + cx * (B[1][cell_index(g, i + 1, j, k)] - B[1][p])
                                           - cy * (B[0][cell_index(g, i, j + 1, k)] - B[0][p]);
            }
}

/* ---------------------------------------------------------------------------
 * Vector-potential formulation (Sec. 4.2).  A sits on the E points; one step
 * advances it by Eq. dadt, A^{n+1/2} = A^{n-1/2} - c dt E^n, with the E^n of the
 * step (call before orc_step).  B = curl_h A on the staggered grid (Eq. viaA,
 * grid form):
 *   Bx[i,j,k] = (Az[i,j,k] - Az[i,j-1,k])/dy - (Ay[i,j,k] - Ay[i,j,k-1])/dz, cyclically;
 * in 2D the z differences vanish.
 * ------------------------------------------------------------------------- */
void orc_update_A(const orc_grid *g, const double *const E[3], double *A[3])
{
    const long long N = (long long)g->nx * g->ny * g->nz;
    for (int a = 0; a < 3; ++a)
        for (long long p = 0; p < N; ++p) A[a][p] -= g->c * g->dt * E[a][p];
}

void orc_curl_A(const orc_grid *g, const double *const A[3], double *B[3])
{
    const double idz = g->dims == 2 ? 0.0 : 1.0 / g->dz;
    for (int k = 0; k < g->nz; ++k)
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i) {
                long long p = cell_index(g, i, j, k);
                B[0][p] = (A[2][p] - A[2][cell_index(g, i, j - 1, k)]) / g->dy -
                          (A[1][p] - A[1][cell_index(g, i, j, k - 1)]) * idz;
                B[1][p] = (A[0][p] - A[0][cell_index(g, i, j, k - 1)]) * idz -
                          (A[2][p] - A[2][cell_index(g, i - 1, j, k)]) / g->dx;
                B[2][p] = (A[1][p] - A[1][cell_index(g, i - 1, j, k)]) / g->dx -
                          (A[0][p] - A[0][cell_index(g, i, j - 1, k)]) / g->dy;
            }
}

/* Generalized momentum of the particles (Sec. 4.2): sum over p of
 * m_p w_p^{n-1/2} + (q_p/c) A^{n-1/2}(x_p^n - (dt/2) u_p^{n-1/2}), with A
 * interpolated by the weights alpha of E (Eq. A) at the time-centred position
 * (in cell units the shift is c_a u_a / (2c) per axis). */
void orc_generalized_momentum(const orc_grid *g, const double *const A[3], int nsp, const orc_species *sp,
                              double P[3])
{
    const double cN[3] = { g->c * g->dt / g->dx, g->c * g->dt / g->dy, g->dims == 2 ? 0.0 : g->c * g->dt / g->dz };
    const long long N = (long long)g->nx * g->ny * g->nz;
    double *zero[3];
    for (int a = 0; a < 3; ++a) zero[a] = (double *)calloc((size_t)N, sizeof(double));
    P[0] = P[1] = P[2] = 0.0;
    for (int s = 0; s < nsp; ++s) {
        const double mp = sp[s].m * sp[s].weight, qp = sp[s].q * sp[s].weight;
        for (long long p = 0; p < sp[s].n; ++p) {
            double w[3] = { sp[s].w[0][p], sp[s].w[1][p], sp[s].w[2][p] };
            double gam = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2] + g->c * g->c);
            double xh[3] = { 0.0, 0.0, 0.0 };
            for (int a = 0; a < g->dims; ++a) {
                double x = sp[s].x[a][p] - 0.5 * cN[a] * w[a] / gam;
                double n = a == 0 ? g->nx : a == 1 ? g->ny : g->nz;
                x = fmod(x, n);
                if (x < 0.0) x += n;
                xh[a] = x;
            }
            double Ap[3], Bp[3];
            orc_gather(g, A, (const double *const *)zero, xh, Ap, Bp);
            for (int a = 0; a < 3; ++a) P[a] += mp * w[a] + qp / g->c * Ap[a];
        }
    }
    for (int a = 0; a < 3; ++a) free(zero[a]);
}

/* ---------------------------------------------------------------------------
 * Particle part of the step for one species (Appendix, step 2): per particle,
 * in storage order, form factor at x^n, gather E and B (B at time n), push,
 * move, deposit, wrap.  Returns the worst deposit closure |sum dF(-)|.
 * ------------------------------------------------------------------------- */
double orc_push_deposit(const orc_grid *g, const double *const E[3], const double *const B[3],
                        double *J[3], orc_species *sp)
{
    const double qm = sp->q / sp->m;
    const double qp = sp->q * sp->weight;
    double worst = 0.0;
    for (long long p = 0; p < sp->n; ++p) {
        double x0[3] = { sp->x[0][p], sp->x[1][p], g->dims == 3 ? sp->x[2][p] : 0.0 };
        double w[3] = { sp->w[0][p], sp->w[1][p], sp->w[2][p] };
        double Ep[3], Bp[3], x1[3], u[3];
        orc_gather(g, E, B, x0, Ep, Bp);
        orc_boris(w, Ep, Bp, qm, g->dt, g->c);
        orc_move(g, w, x0, x1, u);
        double cl = orc_deposit(g, x0, x1, u, qp, J);
        if (cl > worst) worst = cl;
        orc_wrap(g, x1);
        for (int a = 0; a < 3; ++a) sp->w[a][p] = w[a];
        for (int a = 0; a < g->dims; ++a) sp->x[a][p] = x1[a];
    }
    return worst;
}

/* One full time step (Appendix): B half step with E^n; particles; B half step
 * with the same E^n; E full step with J^{n+1/2} and B^{n+1/2}.  J is zeroed
 * first and holds J^{n+1/2} on return.  Returns the worst deposit closure. */
double orc_step(const orc_grid *g, double *E[3], double *B[3], double *J[3], int nsp, orc_species *sp)
{
    const long long N = (long long)g->nx * g->ny * g->nz;
    for (int a = 0; a < 3; ++a) memset(J[a], 0, sizeof(double) * N);
    orc_yee_half_B(g, (const double *const *)E, B);
    double worst = 0.0;
    for (int s = 0; s < nsp; ++s) {
        double cl = orc_push_deposit(g, (const double *const *)E, (const double *const *)B, J, &sp[s]);
        if (cl > worst) worst = cl;
    }
    orc_yee_half_B(g, (const double *const *)E, B);
    orc_yee_E(g, (const double *const *)B, (const double *const *)J, E);
    return worst;
}

/* ---------------------------------------------------------------------------
 * Plane-wave antenna.  The paper motivates laser-plasma runs but gives no
 * injection (reading of the laser setup: a one-way source on a plane of
 * constant x, uniform in y and z).  It is a total-field / scattered-field
 * plane: the incident wave E_inc travels in +x,
 *   E_inc(x, t) = E0 g(tau) sin(omega tau),  tau = t - (x - i0) dx / c,
 *   g(tau) = sin^2(pi tau / (2 ramp)) for 0 < tau < ramp, 1 after, 0 before,
 * with E_y = E_inc, B_z = E_inc (pol 1) or E_z = E_inc, B_y = -E_inc (pol 2).
 * Cells i >= i0 of the B components and i >= i0 of the E components hold the
 * total field, the rest the scattered field.  A B node at x = i0 differences
 * the E node at x = i0 - 1/2, which lacks the incident wave; the E node at
 * x = i0 - 1/2 differences the B node at x = i0, which carries it.  So every
 * B half step of step n (with E at time t^n = n dt) adds, on the plane i = i0,
 *   +(c_x/2) E_inc(i0 - 1/2, t^n) to B_z (pol 1),  -(c_x/2) E_inc(i0 - 1/2, t^n) to B_y (pol 2),
 * and the E step (with B at t^n + dt/2) adds, on the plane i = i0 - 1,
 *   +c_x E_inc(i0, t^n + dt/2) to E_y (pol 1) or to E_z (pol 2)
 * (in both cases minus c_x times the incident B of the B node).
 * ------------------------------------------------------------------------- */
typedef struct {
    int pol;                /* 1: E_y with B_z; 2: E_z with B_y */
    int i0;                 /* first total-field B node along x */
    double E0, omega, ramp; /* amplitude, angular frequency, rise time */
} orc_antenna;

static double orc_incident(const orc_grid *g, const orc_antenna *a, double x, double t)
{
    double tau = t - (x - a->i0) * g->dx / g->c;
    if (tau <= 0.0) return 0.0;
    double env = 1.0;
    if (tau < a->ramp) {
        double s = sin(0.5 * ORC_PI * tau / a->ramp);
        env = s * s;
    }
    return a->E0 * env * sin(a->omega * tau);
}

static void orc_antenna_B(const orc_grid *g, const orc_antenna *a, double t, double *B[3])
{
    const double cx = g->c * g->dt / g->dx;
    const double v = 0.5 * cx * orc_incident(g, a, a->i0 - 0.5, t);
    for (int k = 0; k < g->nz; ++k)
        for (int j = 0; j < g->ny; ++j) {
            long long p = cell_index(g, a->i0, j, k);
            if (a->pol == 1) B[2][p] += v; else B[1][p] -= v;
        }
}

static void orc_antenna_E(const orc_grid *g, const orc_antenna *a, double t, double *E[3])
{
    const double cx = g->c * g->dt / g->dx;
    const double v = cx * orc_incident(g, a, a->i0, t);
    for (int k = 0; k < g->nz; ++k)
        for (int j = 0; j < g->ny; ++j) {
            long long p = cell_index(g, a->i0 - 1, j, k);
            if (a->pol == 1) E[1][p] += v; else E[2][p] += v;
        }
}

/* Step n of a run with an antenna (n counts the steps since the antenna was
 * set): the plain step's sequence with the antenna's sheet terms. */
double orc_step_antenna(const orc_grid *g, const orc_antenna *a, long long n, double *E[3], double *B[3],
                        double *J[3], int nsp, orc_species *sp)
{
    const long long N = (long long)g->nx * g->ny * g->nz;
    const double tn = n * g->dt;
    for (int q = 0; q < 3; ++q) memset(J[q], 0, sizeof(double) * N);
    orc_yee_half_B(g, (const double *const *)E, B);
    orc_antenna_B(g, a, tn, B);
    double worst = 0.0;
    for (int s = 0; s < nsp; ++s) {
        double cl = orc_push_deposit(g, (const double *const *)E, (const double *const *)B, J, &sp[s]);
        if (cl > worst) worst = cl;
    }
    orc_yee_half_B(g, (const double *const *)E, B);
    orc_antenna_B(g, a, tn, B);
    orc_yee_E(g, (const double *const *)B, (const double *const *)J, E);
    orc_antenna_E(g, a, tn + 0.5 * g->dt, E);
    return worst;
}

/* ---------------------------------------------------------------------------
 * Diagnostics at time level n (state E^n, B^{n-1/2}, x^n, w^{n-1/2}):
 *   rho^n from the stored positions (Eq. rho) plus a uniform background;
 *   the Gauss residual r = div_h E - 4 pi rho (Eq. chargelaw; Sec. 2 Poisson form),
 *     div_h E = (Ex[i+1]-Ex[i])/dx + (Ey[j+1]-Ey[j])/dy + (Ez[k+1]-Ez[k])/dz;
 *   the energy integral of Sec. 4.1 summed over particles, with the kinetic part
 *   taken without rest mass and the magnetic energy of B^n = B^{n-1/2} - (1/2)c_h curl E^n;
 *   the particle momentum sum m_p w.
 * rho and resid are outputs of N cells each.
 * ------------------------------------------------------------------------- */
void orc_diagnostics(const orc_grid *g, const double *const E[3], const double *const Bh[3],
                     int nsp, const orc_species *sp, double rho_bg, double *rho, double *resid,
                     orc_diag *out)
{
    const long long N = (long long)g->nx * g->ny * g->nz;
    const double V = cell_volume(g);
    memset(out, 0, sizeof(*out));
    for (long long p = 0; p < N; ++p) rho[p] = 0.0;
    for (int s = 0; s < nsp; ++s)
        orc_rho(g, sp[s].n, (const double *const *)sp[s].x, sp[s].q * sp[s].weight, rho);
    for (long long p = 0; p < N; ++p) rho[p] += rho_bg;
    for (int k = 0; k < g->nz; ++k)
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i) {
                long long p = cell_index(g, i, j, k);
                double div = (E[0][cell_index(g, i + 1, j, k)] - E[0][p]) / g->dx +
                             (E[1][cell_index(g, i, j + 1, k)] - E[1][p]) / g->dy;
                if (g->dims == 3) div += (E[2][cell_index(g, i, j, k + 1)] - E[2][p]) / g->dz;
                resid[p] = div - 4.0 * ORC_PI * rho[p];
                out->charge += V * rho[p];
            }
    double *Bn[3];
    for (int a = 0; a < 3; ++a) {
        Bn[a] = (double *)malloc(sizeof(double) * N);
        memcpy(Bn[a], Bh[a], sizeof(double) * N);
    }
    orc_yee_half_B(g, E, Bn);
    for (long long p = 0; p < N; ++p)
        for (int a = 0; a < 3; ++a) {
            out->field_E += V / (8.0 * ORC_PI) * E[a][p] * E[a][p];
            out->field_B += V / (8.0 * ORC_PI) * Bn[a][p] * Bn[a][p];
        }
    for (int s = 0; s < nsp; ++s) {
        const double mp = sp[s].m * sp[s].weight, qp = sp[s].q * sp[s].weight;
        for (long long p = 0; p < sp[s].n; ++p) {
            double xp[3] = { sp[s].x[0][p], sp[s].x[1][p], g->dims == 3 ? sp[s].x[2][p] : 0.0 };
            double w[3] = { sp[s].w[0][p], sp[s].w[1][p], sp[s].w[2][p] };
            double w2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
            double gam = sqrt(w2 + g->c * g->c);
            out->kinetic += mp * g->c * (gam - g->c);
            double Ep[3], Bp[3];
            orc_gather(g, E, (const double *const *)Bn, xp, Ep, Bp);
            for (int a = 0; a < 3; ++a) {
                out->half_step_corr += 0.5 * qp * g->dt * (g->c * w[a] / gam) * Ep[a];
                out->momentum[a] += mp * w[a];
            }
        }
    }
    out->total = out->kinetic + out->field_E + out->field_B + out->half_step_corr;
    for (int a = 0; a < 3; ++a) free(Bn[a]);
}

/* ---------------------------------------------------------------------------
 * Tile sort.  The key of a particle is the linear index of the tile that holds
 * its cell: tile (ti, tj, tk) = (i/Tx, j/Ty, k/Tz), key = (tk*nty + tj)*ntx + ti
 * with nt_a = ceil(n_a/T_a).  The permutation is the stable counting sort by
 * key: perm[o] is the input index that lands at output slot o; equal keys keep
 * their input order.
 * ------------------------------------------------------------------------- */
void orc_tile_keys(const orc_grid *g, const int tile[3], long long n, const double *const x[3], int *key)
{
    const long long ntx = (g->nx + tile[0] - 1) / tile[0];
    const long long nty = (g->ny + tile[1] - 1) / tile[1];
    for (long long p = 0; p < n; ++p) {
        long long i = (long long)floor(x[0][p]), j = (long long)floor(x[1][p]);
        long long k = g->dims == 3 ? (long long)floor(x[2][p]) : 0;
        long long tk = g->dims == 3 ? k / tile[2] : 0;
        key[p] = (int)((tk * nty + j / tile[1]) * ntx + i / tile[0]);
    }
}

int orc_sort_perm(long long n, const int *key, int nkeys, long long *perm)
{
    long long *start = (long long *)calloc((size_t)nkeys + 1, sizeof(long long));
    if (!start) return -1;
    for (long long p = 0; p < n; ++p) {
        if (key[p] < 0 || key[p] >= nkeys) { free(start); return -2; }
        start[key[p] + 1] += 1;
    }
    for (int t = 0; t < nkeys; ++t) start[t + 1] += start[t];
    for (long long p = 0; p < n; ++p) perm[start[key[p]]++] = p;
    free(start);
    return 0;
}

/* ===========================================================================
 * Discrete adjoint of one time step (hand-derived reverse mode of the
 * Appendix step above), for l_a = 1 1/2.  State at level n: E^n, B^{n-1/2}, x^n, w^{n-1/2};
 * the adjoints lam* hold dL/d(state at n+1) on entry and dL/d(state at n) on
 * return.  The step's intermediate quantities are recomputed from the state at
 * n.  Forward order: B1 = B - (1/2) C_B E; particles (gather from E, B1; push;
 * move; deposit into J); B2 = B1 - (1/2) C_B E; E' = E - 4 pi dt J + C_E B2.
 * Reverse order: transpose of the E step, of the second B half step, of every
 * particle, of the first B half step.  Cell indices (floor) are piecewise
 * constant and contribute no derivative.
 * ========================================================================= */

/* derivatives of the l_a = 1 1/2 values with respect to x_p (d = x_p - i) */
static void form_factor_deriv(double xp, double df[2], double dS[3])
{
    double d = xp - floor(xp);
    df[0] = -1.0;
    df[1] = 1.0;
    dS[0] = -(1.0 - d);
    dS[1] = 1.0 - 2.0 * d;
    dS[2] = d;
}

/* Transpose of B -= (1/2) curl_h E (orc_yee_half_B): lamE += (-(1/2) C_B)^T lamB. */
void orc_yee_half_B_adj(const orc_grid *g, const double *const lamB[3], double *lamE[3])
{
    const double cx = g->c * g->dt / g->dx, cy = g->c * g->dt / g->dy;
    const double cz = g->dims == 2 ? 0.0 : g->c * g->dt / g->dz;
    for (int k = 0; k < g->nz; ++k)
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i) {
                long long p = cell_index(g, i, j, k);
                /* Bx[p] = ... - 0.5 cy (Ez[p] - Ez[j-1]) + 0.5 cz (Ey[p] - Ey[k-1]) */
                lamE[2][p] += -0.5 * cy * lamB[0][p];
                lamE[2][cell_index(g, i, j - 1, k)] += 0.5 * cy * lamB[0][p];
                lamE[1][p] += 0.5 * cz * lamB[0][p];
                lamE[1][cell_index(g, i, j, k - 1)] += -0.5 * cz * lamB[0][p];
                /* By[p] = ... - 0.5 cz (Ex[p] - Ex[k-1]) + 0.5 cx (Ez[p] - Ez[i-1]) */
                lamE[0][p] += -0.5 * cz * lamB[1][p];
                lamE[0][cell_index(g, i, j, k - 1)] += 0.5 * cz * lamB[1][p];
                lamE[2][p] += 0.5 * cx * lamB[1][p];
                lamE[2][cell_index(g, i - 1, j, k)] += -0.5 * cx * lamB[1][p];
                /* Bz[p] = ... - 0.5 cx (Ey[p] - Ey[i-1]) + 0.5 cy (Ex[p] - Ex[j-1]) */
                lamE[1][p] += -0.5 * cx * lamB[2][p];
                lamE[1][cell_index(g, i - 1, j, k)] += 0.5 * cx * lamB[2][p];
                lamE[0][p] += 0.5 * cy * lamB[2][p];
                lamE[0][cell_index(g, i, j - 1, k)] += -0.5 * cy * lamB[2][p];
            }
}

/* Transpose of E += -4 pi dt J + C_E B (orc_yee_E): lamE passes through,
 * lamB += C_E^T lamE, lamJ = -4 pi dt lamE. */
void orc_yee_E_adj(const orc_grid *g, const double *const lamE[3], double *lamB[3], double *lamJ[3])
{
    const double cx = g->c * g->dt / g->dx, cy = g->c * g->dt / g->dy;
    const double cz = g->dims == 2 ? 0.0 : g->c * g->dt / g->dz;
    const double fpdt = 4.0 * ORC_PI * g->dt;
    for (int k = 0; k < g->nz; ++k)
        for (int j = 0; j < g->ny; ++j)
            for (int i = 0; i < g->nx; ++i) {
                long long p = cell_index(g, i, j, k);
                for (int a = 0; a < 3; ++a) lamJ[a][p] = -fpdt * lamE[a][p];
                /* Ex[p] += cy (Bz[j+1] - Bz[p]) - cz (By[k+1] - By[p]) */
                lamB[2][cell_index(g, i, j + 1, k)] += cy * lamE[0][p];
                lamB[2][p] += -cy * lamE[0][p];
                lamB[1][cell_index(g, i, j, k + 1)] += -cz * lamE[0][p];
                lamB[1][p] += cz * lamE[0][p];
                /* Ey[p] += cz (Bx[k+1] - Bx[p]) - cx (Bz[i+1] - Bz[p]) */
                lamB[0][cell_index(g, i, j, k + 1)] += cz * lamE[1][p];
                lamB[0][p] += -cz * lamE[1][p];
                lamB[2][cell_index(g, i + 1, j, k)] += -cx * lamE[1][p];
                lamB[2][p] += cx * lamE[1][p];
                /* Ez[p] += cx (By[i+1] - By[p]) - cy (Bx[j+1] - Bx[p]) */
                lamB[1][cell_index(g, i + 1, j, k)] += cx * lamE[2][p];
                lamB[1][p] += -cx * lamE[2][p];
                lamB[0][cell_index(g, i, j + 1, k)] += -cy * lamE[2][p];
                lamB[0][p] += cy * lamE[2][p];
            }
}

/* Transpose of the gather (orc_gather) at x_p: scatter lamEp alpha into lamE and
 * lamBp beta into lamB, and add sum (d alpha/d x_p) E lamEp + (d beta/d x_p) B lamBp
 * to lam_x. */
void orc_gather_adj(const orc_grid *g, const double *const E[3], const double *const B[3], const double xp[3],
                    const double lamEp[3], const double lamBp[3], double *lamE[3], double *lamB[3], double lam_x[3])
{
    orc_weights wt;
    particle_weights(g, xp, &wt);
    double dw[3][2][3];   /* [axis][0: d f, 1: d dF][index] */
    for (int a = 0; a < 3; ++a) {
        double df[2], dS[3];
        if (a == 2 && g->dims == 2) {
            df[0] = df[1] = 0.0;
            dS[0] = dS[1] = dS[2] = 0.0;
        } else {
            form_factor_deriv(xp[a], df, dS);
        }
        dw[a][0][0] = df[0]; dw[a][0][1] = df[1]; dw[a][0][2] = 0.0;
        dw[a][1][0] = dS[0]; dw[a][1][1] = dS[1]; dw[a][1][2] = dS[2];
    }
    const long long i0[3] = { wt.ax[0].ib, wt.ax[1].ib, wt.ax[2].ib };
    /* per component: which family (0 = f at integer points, 1 = dF at half-integers) per axis */
    const int famE[3][3] = { { 0, 1, 1 }, { 1, 0, 1 }, { 1, 1, 0 } };
    const int famB[3][3] = { { 1, 0, 0 }, { 0, 1, 0 }, { 0, 0, 1 } };
    for (int fld = 0; fld < 2; ++fld)
        for (int c = 0; c < 3; ++c) {
            const int *fam = fld == 0 ? famE[c] : famB[c];
            const double lam = fld == 0 ? lamEp[c] : lamBp[c];
            const double *F = fld == 0 ? E[c] : B[c];
            double *LF = fld == 0 ? lamE[c] : lamB[c];
            int cnt[3], off[3];
            for (int a = 0; a < 3; ++a) {
                if (a == 2 && g->dims == 2) { cnt[a] = 1; off[a] = 0; continue; }
                cnt[a] = fam[a] == 0 ? 2 : 3;
                off[a] = fam[a] == 0 ? 0 : -1;
            }
            for (int s2 = 0; s2 < cnt[2]; ++s2)
                for (int s1 = 0; s1 < cnt[1]; ++s1)
                    for (int s0 = 0; s0 < cnt[0]; ++s0) {
                        const int sidx[3] = { s0, s1, s2 };
                        double v[3], d[3];
                        for (int a = 0; a < 3; ++a) {
                            if (a == 2 && g->dims == 2) { v[a] = 1.0; d[a] = 0.0; continue; }
                            if (fam[a] == 0) { v[a] = wt.ax[a].f[sidx[a]]; d[a] = dw[a][0][sidx[a]]; }
                            else { v[a] = wt.ax[a].dF[sidx[a]]; d[a] = dw[a][1][sidx[a]]; }
                        }
                        long long idx = cell_index(g, i0[0] + off[0] + s0, i0[1] + off[1] + s1,
                                                   i0[2] + off[2] + s2);
                        LF[idx] += v[0] * v[1] * v[2] * lam;
                        lam_x[0] += d[0] * v[1] * v[2] * F[idx] * lam;
                        lam_x[1] += v[0] * d[1] * v[2] * F[idx] * lam;
                        lam_x[2] += v[0] * v[1] * d[2] * F[idx] * lam;
                    }
        }
}

/* Transpose of orc_boris: given the pre-push w, Ep, Bp and lam_w1 = dL/dw^{n+1/2},
 * return lam_w0 = dL/dw^{n-1/2}, lamEp, lamBp (the push's reverse sweep). */
void orc_boris_adj(const double w[3], const double Ep[3], const double Bp[3], double qm, double dt, double c,
                   const double lam_w1[3], double lam_w0[3], double lamEp[3], double lamBp[3])
{
    const double h = 0.5 * qm * dt;
    double e[3], t[3], b[3], n[3], m[3], tb[3];
    for (int a = 0; a < 3; ++a) e[a] = h * Ep[a];
    for (int a = 0; a < 3; ++a) t[a] = w[a] + e[a];
    double gt = sqrt(t[0] * t[0] + t[1] * t[1] + t[2] * t[2] + c * c);
    double s = h / gt;
    for (int a = 0; a < 3; ++a) b[a] = s * Bp[a];
    cross(t, b, tb);
    for (int a = 0; a < 3; ++a) n[a] = t[a] + tb[a];
    double b2 = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
    double F = 2.0 / (1.0 + b2);
    cross(n, b, m);
    /* w1 = t + e + F m */
    double lt[3], le[3], lm[3], ln[3], lb[3], tmp[3];
    double lF = 0.0;
    for (int a = 0; a < 3; ++a) {
        lt[a] = lam_w1[a];
        le[a] = lam_w1[a];
        lm[a] = F * lam_w1[a];
        lF += lam_w1[a] * m[a];
    }
    /* m = n x b:  d(lm.(n x b))/dn = b x lm,  /db = lm x n */
    cross(b, lm, ln);
    cross(lm, n, lb);
    /* F = 2/(1+b2), b2 = b.b */
    double lb2 = lF * (-2.0 / ((1.0 + b2) * (1.0 + b2)));
    for (int a = 0; a < 3; ++a) lb[a] += 2.0 * b[a] * lb2;
    /* n = t + t x b */
    cross(b, ln, tmp);
    for (int a = 0; a < 3; ++a) lt[a] += ln[a] + tmp[a];
    cross(ln, t, tmp);
    for (int a = 0; a < 3; ++a) lb[a] += tmp[a];
    /* b = s Bp, s = h/gt, gt = sqrt(t.t + c^2) */
    double ls = 0.0;
    for (int a = 0; a < 3; ++a) {
        ls += lb[a] * Bp[a];
        lamBp[a] = s * lb[a];
    }
    double lgt = -ls * h / (gt * gt);
    for (int a = 0; a < 3; ++a) lt[a] += lgt * t[a] / gt;
    /* t = w + e, e = h Ep */
    for (int a = 0; a < 3; ++a) {
        lam_w0[a] = lt[a];
        le[a] += lt[a];
        lamEp[a] = h * le[a];
    }
}

/* Window of one axis of the deposit together with the derivatives of the placed
 * old/new weights with respect to x^n (dold) and x^{n+1} (dnew). */
typedef struct {
    orc_axis_current cur;
    double old_w[ORC_MAXWIN], new_w[ORC_MAXWIN];
    double dold[ORC_MAXWIN], dnew[ORC_MAXWIN];
} orc_axis_adj;

static int axis_current_adj(double x0, double x1, orc_axis_adj *ad)
{
    if (axis_current(3, x0, x1, &ad->cur) != 0) return -1;
    long long i0, i1;
    double f0[2], f1[2], dF0[3], dF1[3], df[2], dS0[3], dS1[3];
    orc_form_factor(x0, &i0, f0, dF0);
    orc_form_factor(x1, &i1, f1, dF1);
    form_factor_deriv(x0, df, dS0);
    form_factor_deriv(x1, df, dS1);
    const long long lo = ad->cur.lo;
    for (int s = 0; s < ad->cur.len; ++s) {
        ad->old_w[s] = ad->new_w[s] = ad->dold[s] = ad->dnew[s] = 0.0;
    }
    for (int b = 0; b < 3; ++b) {
        ad->old_w[i0 - 1 + b - lo] = dF0[b];
        ad->dold[i0 - 1 + b - lo] = dS0[b];
        ad->new_w[i1 - 1 + b - lo] = dF1[b];
        ad->dnew[i1 - 1 + b - lo] = dS1[b];
    }
    return 0;
}

/* Transpose of orc_deposit: given lamJ (grid), return the contributions to
 * lam_x0, lam_x1 and lam_u (u enters the 2D z current only). */
void orc_deposit_adj(const orc_grid *g, const double x0[3], const double x1[3], const double u[3], double qp,
                     const double *const lamJ[3], double lam_x0[3], double lam_x1[3], double lam_u[3])
{
    orc_axis_adj ax[3];
    double lPp[3][ORC_MAXWIN], lPm[3][ORC_MAXWIN], lD[3][ORC_MAXWIN];
    for (int a = 0; a < g->dims; ++a) {
        if (axis_current_adj(x0[a], x1[a], &ax[a]) != 0) return;
        for (int s = 0; s < ORC_MAXWIN; ++s) lPp[a][s] = lPm[a][s] = lD[a][s] = 0.0;
    }
    const double qV = qp / cell_volume(g);
    const double dtn = g->dt;
    if (g->dims == 3) {
        /* xi^(a) on faces of axis a: k_a D_a(f) [Pp_b Pp_c + Pm_b Pm_c / 3], (b, c) the two other axes */
        const double dd[3] = { g->dx, g->dy, g->dz };
        for (int a = 0; a < 3; ++a) {
            const int b = (a + 1) % 3, cax = (a + 2) % 3;
            const double ka = -0.25 * (dd[a] / dtn) * qV;
            const orc_axis_current *A = &ax[a].cur, *Bc = &ax[b].cur, *Cc = &ax[cax].cur;
            for (int sc = 0; sc < Cc->len; ++sc)
                for (int sb = 0; sb < Bc->len; ++sb)
                    for (int sa = 1; sa < A->len; ++sa) {
                        long long idx[3];
                        idx[a] = A->lo + sa;
                        idx[b] = Bc->lo + sb;
                        idx[cax] = Cc->lo + sc;
                        const double G = lamJ[a][cell_index(g, idx[0], idx[1], idx[2])] * ka;
                        const double T = Bc->Pp[sb] * Cc->Pp[sc] + Bc->Pm[sb] * Cc->Pm[sc] / 3.0;
                        lD[a][sa] += G * T;
                        lPp[b][sb] += G * A->D[sa] * Cc->Pp[sc];
                        lPp[cax][sc] += G * A->D[sa] * Bc->Pp[sb];
                        lPm[b][sb] += G * A->D[sa] * Cc->Pm[sc] / 3.0;
                        lPm[cax][sc] += G * A->D[sa] * Bc->Pm[sb] / 3.0;
                    }
        }
    } else {
        const orc_axis_current *X = &ax[0].cur, *Y = &ax[1].cur;
        const double kx = -0.5 * (g->dx / dtn) * qV, ky = -0.5 * (g->dy / dtn) * qV, kz = 0.25 * qV;
        for (int sj = 0; sj < Y->len; ++sj)
            for (int si = 1; si < X->len; ++si) {
                const double G = lamJ[0][cell_index(g, X->lo + si, Y->lo + sj, 0)] * kx;
                lD[0][si] += G * Y->Pp[sj];
                lPp[1][sj] += G * X->D[si];
            }
        for (int sj = 1; sj < Y->len; ++sj)
            for (int si = 0; si < X->len; ++si) {
                const double G = lamJ[1][cell_index(g, X->lo + si, Y->lo + sj, 0)] * ky;
                lD[1][sj] += G * X->Pp[si];
                lPp[0][si] += G * Y->D[sj];
            }
        for (int sj = 0; sj < Y->len; ++sj)
            for (int si = 0; si < X->len; ++si) {
                const double G = lamJ[2][cell_index(g, X->lo + si, Y->lo + sj, 0)] * kz;
                lam_u[2] += G * (X->Pp[si] * Y->Pp[sj] + X->Pm[si] * Y->Pm[sj] / 3.0);
                lPp[0][si] += G * u[2] * Y->Pp[sj];
                lPp[1][sj] += G * u[2] * X->Pp[si];
                lPm[0][si] += G * u[2] * Y->Pm[sj] / 3.0;
                lPm[1][sj] += G * u[2] * X->Pm[si] / 3.0;
            }
    }
    for (int a = 0; a < g->dims; ++a) {
        const orc_axis_current *A = &ax[a].cur;
        /* D(f) = sum_{s < f} Pm(s): lam Pm(s) += sum_{f > s} lam D(f) */
        for (int s = 0; s < A->len; ++s)
            for (int f = s + 1; f < A->len; ++f) lPm[a][s] += lD[a][f];
        for (int s = 0; s < A->len; ++s) {
            const double lnew = lPp[a][s] + lPm[a][s];   /* Pp = new + old, Pm = new - old */
            const double lold = lPp[a][s] - lPm[a][s];
            lam_x1[a] += lnew * ax[a].dnew[s];
            lam_x0[a] += lold * ax[a].dold[s];
        }
    }
}

/* One step of the adjoint (see the block comment above).  The species' x and w
 * are the state at level n and are not modified; lam_x[s][a], lam_w[s][a] are the
 * per-particle adjoints of species s. */
void orc_step_adj(const orc_grid *g, const double *const E[3], const double *const Bh[3], int nsp,
                  const orc_species *sp, double *lamE[3], double *lamB[3], double *const *lam_x,
                  double *const *lam_w)
{
    if (grid_order2(g) != 3) return;   /* the hand-derived adjoint is written for l_a = 1 1/2 */
    const long long N = (long long)g->nx * g->ny * g->nz;
    double *B1[3], *lamJ[3], *lamB1[3];
    for (int a = 0; a < 3; ++a) {
        B1[a] = (double *)malloc(sizeof(double) * N);
        lamJ[a] = (double *)calloc(N, sizeof(double));
        lamB1[a] = (double *)calloc(N, sizeof(double));
        memcpy(B1[a], Bh[a], sizeof(double) * N);
    }
    orc_yee_half_B(g, E, B1);
    /* (E step)^T: lamE unchanged, lamB (= lam B2) += C_E^T lamE, lamJ */
    orc_yee_E_adj(g, (const double *const *)lamE, lamB, lamJ);
    /* (second B half step)^T: lam B1 = lam B2, lamE += (-C_B/2)^T lam B2 */
    orc_yee_half_B_adj(g, (const double *const *)lamB, lamE);
    for (int a = 0; a < 3; ++a) memcpy(lamB1[a], lamB[a], sizeof(double) * N);
    /* particles^T */
    const double cN[3] = { g->c * g->dt / g->dx, g->c * g->dt / g->dy, g->c * g->dt / g->dz };
    for (int s = 0; s < nsp; ++s) {
        const double qm = sp[s].q / sp[s].m, qp = sp[s].q * sp[s].weight;
        for (long long p = 0; p < sp[s].n; ++p) {
            double x0[3] = { sp[s].x[0][p], sp[s].x[1][p], g->dims == 3 ? sp[s].x[2][p] : 0.0 };
            double w0[3] = { sp[s].w[0][p], sp[s].w[1][p], sp[s].w[2][p] };
            double Ep[3], Bp[3], w1[3], x1[3], u[3];
            orc_gather(g, E, (const double *const *)B1, x0, Ep, Bp);
            for (int a = 0; a < 3; ++a) w1[a] = w0[a];
            orc_boris(w1, Ep, Bp, qm, g->dt, g->c);
            orc_move(g, w1, x0, x1, u);
            double lx0[3] = { 0, 0, 0 }, lx1[3], lu[3] = { 0, 0, 0 }, lw1[3];
            for (int a = 0; a < 3; ++a) {
                lx1[a] = a < g->dims ? lam_x[s][a * sp[s].n + p] : 0.0;
                lw1[a] = lam_w[s][a * sp[s].n + p];
            }
            orc_deposit_adj(g, x0, x1, u, qp, (const double *const *)lamJ, lx0, lx1, lu);
            /* x1 = x0 + cN w1/gamma1;  u = c w1/gamma1 */
            const double gam = sqrt(w1[0] * w1[0] + w1[1] * w1[1] + w1[2] * w1[2] + g->c * g->c);
            for (int a = 0; a < g->dims; ++a) lx0[a] += lx1[a];
            for (int b = 0; b < 3; ++b) {
                double acc = 0.0;
                for (int a = 0; a < 3; ++a) {
                    const double jac = ((a == b ? 1.0 : 0.0) / gam - w1[a] * w1[b] / (gam * gam * gam));
                    if (a < g->dims) acc += lx1[a] * cN[a] * jac;
                    acc += lu[a] * g->c * jac;
                }
                lw1[b] += acc;
            }
            double lw0[3], lEp[3], lBp[3];
            orc_boris_adj(w0, Ep, Bp, qm, g->dt, g->c, lw1, lw0, lEp, lBp);
            orc_gather_adj(g, E, (const double *const *)B1, x0, lEp, lBp, lamE, lamB1, lx0);
            for (int a = 0; a < 3; ++a) {
                if (a < g->dims) lam_x[s][a * sp[s].n + p] = lx0[a];
                lam_w[s][a * sp[s].n + p] = lw0[a];
            }
        }
    }
    /* (first B half step)^T: lam B = lam B1, lamE += (-C_B/2)^T lam B1 */
    orc_yee_half_B_adj(g, (const double *const *)lamB1, lamE);
    for (int a = 0; a < 3; ++a) {
        memcpy(lamB[a], lamB1[a], sizeof(double) * N);
        free(B1[a]);
        free(lamJ[a]);
        free(lamB1[a]);
    }
}

/*
 * w1_oracle.c -- plain, slow FP64 CPU restatement of the multilevel primal-dual
 * Wasserstein-1 solver of Liu, Yin, Li and Chow, "Multilevel Optimal Transport:
 * a Fast Approximation of Wasserstein-1 distances" (arXiv 1810.00118).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the reference the CUDA path is checked
 * against.  Only the test-suite, the smoke check and the benchmark's CPU-baseline
 * leg may load it.  It shares no code, header, table or helper with the CUDA
 * library, and the CUDA library never calls it.
 *
 * Everything is FP64, single-threaded, written as plain loops in the order the
 * paper states the method, so that it can be checked against the paper by eye.
 *
 * Grid and layout (the reading of Sec. 2.2 used throughout; the paper's vertex
 * grid {0,h,...,1}^d cannot be nested 2:1 with 512 nodes per side, so the nodes
 * are pixel centres and the levels are nested by 2x2 agglomeration):
 *   - nx * ny nodes, spacing h, node (i, j) with i along x_1, j along x_2;
 *   - every plane is row-major [j][i], index j*nx + i;
 *   - m1[j][i] is the flux on the x-edge (i,j)->(i+1,j); m1[j][nx-1] does not
 *     exist (zero-flux boundary) and is kept at 0;
 *   - m2[j][i] is the flux on the y-edge (i,j)->(i,j+1); m2[ny-1][i] is kept at 0.
 *
 * Parity pins: every exported function is pinned by tests that do not retype
 * it (exact LP / min-cost flow on small grids, the 1-D closed form, translated
 * bumps, adjoint and commutation identities, Lemma 3.1, brute force on 2x2).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define W1O_NORM_L1 1
#define W1O_NORM_L2 2
#define W1O_NORM_LINF 3

#define W1O_STOP_GAP 0
#define W1O_STOP_FPR 1

#define W1O_OK 0
#define W1O_NOT_CONVERGED 1
#define W1O_ERR_ARG (-1)
#define W1O_ERR_SHAPE (-2)
#define W1O_ERR_MASS (-3)
#define W1O_ERR_NOMEM (-4)

/* Statistics of one state (m, phi) on one level.  The field order is part of
 * the Python binding (oracle/__init__.py). */
typedef struct {
    double f;      /* f(m) = sum_x ||m(x)||_p h^2, the primal objective (eq. opt_flux_dis) */
    double dual;   /* D(phi) = -<phi, rho>_h, the dual objective of eq. opt_dual3 (sign: see w1o_stats) */
    double res_l1; /* sum_x |rho(x) - div m(x)| h^2 */
    double rho_l1; /* sum_x |rho(x)| h^2 */
    double gmax;   /* max_x ||grad phi(x)||_q, q the dual exponent of p */
    double lb;     /* certified lower bound D(phi) / max(1, gmax) */
    double route;  /* cost of an explicit flux that carries the residual rho - div m */
    double ub;     /* certified upper bound f(m) + route */
    double fpr;    /* fixed-point residual R^k of eq. pd_stop for the step out of this state */
    double saddle; /* L(m, phi) = f(m) + <phi, A m - rho>_h, the Lagrangian of eq. minmax_cp */
} w1o_stats_t;

#define AT(a, j, i) ((a)[(size_t)(j) * (size_t)nx + (size_t)(i)])

/* ------------------------------------------------------------------------- */
/* Operators of Sec. 2.2                                                      */
/* ------------------------------------------------------------------------- */

/* Discrete divergence div^h = A_h of Sec. 2.2 (the case formula for D_{h,i}):
 *   x_i at the first node : m_i(x)/h
 *   interior             : (m_i(x) - m_i(x - h e_i))/h
 *   x_i at the last node : -m_i(x - h e_i)/h     (printed "x_i > 1", read "x_i = 1")
 * The flux component at the last node of its own direction is not a variable
 * (zero-flux boundary), so it is never read. */
void w1o_div(int nx, int ny, double h, const double* m1, const double* m2, double* out)
{
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            double d1 = 0.0, d2 = 0.0;
            if (i < nx - 1) d1 += AT(m1, j, i);
            if (i > 0) d1 -= AT(m1, j, i - 1);
            if (j < ny - 1) d2 += AT(m2, j, i);
            if (j > 0) d2 -= AT(m2, j - 1, i);
            AT(out, j, i) = d1 / h + d2 / h;
        }
    }
}

/* Forward-difference gradient, the negative adjoint of div^h (A_h^* in
 * eq. opt_dual3 is -grad): <phi, div m>_h = -<grad phi, m>_h for every flux m.
 * Components that would leave the grid are 0. */
void w1o_grad(int nx, int ny, double h, const double* phi, double* g1, double* g2)
{
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            AT(g1, j, i) = (i < nx - 1) ? (AT(phi, j, i + 1) - AT(phi, j, i)) / h : 0.0;
            AT(g2, j, i) = (j < ny - 1) ? (AT(phi, j + 1, i) - AT(phi, j, i)) / h : 0.0;
        }
    }
}

/* Euclidean projection of (u1, u2) onto the unit l1 ball {|a| + |b| <= 1}:
 * soft thresholding by the lambda >= 0 that makes the l1 norm exactly 1. */
static void proj_l1_ball(double u1, double u2, double* p1, double* p2)
{
    double a = fabs(u1), b = fabs(u2);
    if (a + b <= 1.0) {
        *p1 = u1;
        *p2 = u2;
        return;
    }
    /* sum_i max(|u_i| - lambda, 0) = 1 */
    double lambda;
    if (a - b >= 1.0) lambda = a - 1.0;
    else if (b - a >= 1.0) lambda = b - 1.0;
    else lambda = 0.5 * (a + b - 1.0);
    double r1 = a - lambda, r2 = b - lambda;
    *p1 = r1 > 0.0 ? copysign(r1, u1) : 0.0;
    *p2 = r2 > 0.0 ? copysign(r2, u2) : 0.0;
}

/* Proximal map of mu*||.||_p at one node, the closed form of the argmin in the
 * first line of eq. primaldual (p = 1: componentwise soft threshold; p = 2:
 * shrink the vector's length by mu; p = infinity: by the Moreau decomposition
 * named in Sec. 4, v - mu * Proj_{l1 ball}(v / mu), the l1 ball being the unit
 * ball of the dual norm). */
static void prox_node(int norm, double mu, double v1, double v2, double* o1, double* o2)
{
    if (norm == W1O_NORM_L1) {
        double a1 = fabs(v1) - mu, a2 = fabs(v2) - mu;
        *o1 = a1 > 0.0 ? copysign(a1, v1) : 0.0;
        *o2 = a2 > 0.0 ? copysign(a2, v2) : 0.0;
    } else if (norm == W1O_NORM_LINF) {
        double p1, p2;
        proj_l1_ball(v1 / mu, v2 / mu, &p1, &p2);
        *o1 = v1 - mu * p1;
        *o2 = v2 - mu * p2;
    } else {
        double len = sqrt(v1 * v1 + v2 * v2);
        double s = (len > mu) ? 1.0 - mu / len : 0.0;
        *o1 = v1 * s;
        *o2 = v2 * s;
    }
}

void w1o_prox(int norm, double mu, int n, const double* v1, const double* v2, double* o1, double* o2)
{
    for (int k = 0; k < n; ++k) prox_node(norm, mu, v1[k], v2[k], &o1[k], &o2[k]);
}

/* ||m(x)||_p at one node */
static double node_norm(int norm, double a, double b)
{
    if (norm == W1O_NORM_L1) return fabs(a) + fabs(b);
    if (norm == W1O_NORM_LINF) return fmax(fabs(a), fabs(b));
    return sqrt(a * a + b * b);
}

/* ||g||_q at one node, 1/p + 1/q = 1: q = infinity for p = 1, 2 for 2, 1 for infinity */
static double node_dual_norm(int norm, double a, double b)
{
    if (norm == W1O_NORM_L1) return fmax(fabs(a), fabs(b));
    if (norm == W1O_NORM_LINF) return fabs(a) + fabs(b);
    return sqrt(a * a + b * b);
}

/* ------------------------------------------------------------------------- */
/* Algorithm 1: one step of eq. primaldual                                    */
/* ------------------------------------------------------------------------- */

typedef struct {
    int nx, ny;
    double *g1, *g2, *n1, *n2, *b1, *b2, *d, *dphi, *dm1, *dm2, *ddiv;
} scratch_t;

static int scratch_alloc(scratch_t* s, int nx, int ny)
{
    size_t n = (size_t)nx * (size_t)ny;
    memset(s, 0, sizeof(*s));
    s->nx = nx;
    s->ny = ny;
    double** f[] = {&s->g1, &s->g2, &s->n1, &s->n2, &s->b1, &s->b2, &s->d, &s->dphi, &s->dm1, &s->dm2, &s->ddiv};
    for (size_t k = 0; k < sizeof(f) / sizeof(f[0]); ++k) {
        *f[k] = (double*)calloc(n ? n : 1, sizeof(double));
        if (!*f[k]) return W1O_ERR_NOMEM;
    }
    return W1O_OK;
}

static void scratch_free(scratch_t* s)
{
    free(s->g1); free(s->g2); free(s->n1); free(s->n2); free(s->b1); free(s->b2);
    free(s->d); free(s->dphi); free(s->dm1); free(s->dm2); free(s->ddiv);
    memset(s, 0, sizeof(*s));
}

/* One iteration of eq. primaldual.  With L(m, phi) = f(m) + <phi, div m - rho>_h
 * and the L2 metrics of Sec. 2.2, every h^2 weight cancels and the three lines
 * read
 *     m^{k+1}   = prox_{mu ||.||_p}( m^k + mu * grad phi^k )
 *     mbar      = 2 m^{k+1} - m^k
 *     phi^{k+1} = phi^k + tau * ( div mbar - rho ).
 * If fpr is not NULL it receives R^k of eq. pd_stop for this step. */
static void cp_step(scratch_t* s, double h, int norm, double mu, double tau, const double* rho,
                    double* m1, double* m2, double* phi, double* fpr)
{
    const int nx = s->nx, ny = s->ny;
    const size_t n = (size_t)nx * (size_t)ny;
    /* primal: m^{k+1} = argmin_m L(m, phi^k) + ||m - m^k||^2_{L2} / (2 mu) */
    w1o_grad(nx, ny, h, phi, s->g1, s->g2);
    for (size_t k = 0; k < n; ++k)
        prox_node(norm, mu, m1[k] + mu * s->g1[k], m2[k] + mu * s->g2[k], &s->n1[k], &s->n2[k]);
    /* the boundary flux is not a variable */
    for (int j = 0; j < ny; ++j) AT(s->n1, j, nx - 1) = 0.0;
    for (int i = 0; i < nx; ++i) AT(s->n2, ny - 1, i) = 0.0;
    /* extrapolation: mbar = 2 m^{k+1} - m^k */
    for (size_t k = 0; k < n; ++k) {
        s->b1[k] = 2.0 * s->n1[k] - m1[k];
        s->b2[k] = 2.0 * s->n2[k] - m2[k];
    }
    /* dual: phi^{k+1} = argmax_phi L(mbar, phi) - ||phi - phi^k||^2_{L2} / (2 tau) */
    w1o_div(nx, ny, h, s->b1, s->b2, s->d);
    for (size_t k = 0; k < n; ++k) s->dphi[k] = tau * (s->d[k] - rho[k]);
    if (fpr) {
        /* R^k = ||dm||^2_{L2}/mu + ||dphi||^2_{L2}/tau - 2 <dphi, A dm>_h  (eq. pd_stop) */
        for (size_t k = 0; k < n; ++k) {
            s->dm1[k] = s->n1[k] - m1[k];
            s->dm2[k] = s->n2[k] - m2[k];
        }
        w1o_div(nx, ny, h, s->dm1, s->dm2, s->ddiv);
        double a = 0.0, b = 0.0, c = 0.0;
        for (size_t k = 0; k < n; ++k) {
            a += s->dm1[k] * s->dm1[k] + s->dm2[k] * s->dm2[k];
            b += s->dphi[k] * s->dphi[k];
            c += s->dphi[k] * s->ddiv[k];
        }
        *fpr = (a / mu + b / tau - 2.0 * c) * h * h;
    }
    for (size_t k = 0; k < n; ++k) {
        phi[k] += s->dphi[k];
        m1[k] = s->n1[k];
        m2[k] = s->n2[k];
    }
}

/* Run `iters` steps of eq. primaldual in place; *fpr (if not NULL) gets R^k of
 * the last step. */
int w1o_cp_iterate(int nx, int ny, double h, int norm, double mu, double tau, const double* rho,
                   double* m1, double* m2, double* phi, long iters, double* fpr)
{
    if (nx < 1 || ny < 1 || !(h > 0.0)) return W1O_ERR_ARG;
    scratch_t s;
    if (scratch_alloc(&s, nx, ny) != W1O_OK) {
        scratch_free(&s);
        return W1O_ERR_NOMEM;
    }
    for (long k = 0; k < iters; ++k) cp_step(&s, h, norm, mu, tau, rho, m1, m2, phi, (k == iters - 1) ? fpr : NULL);
    scratch_free(&s);
    return W1O_OK;
}

/* ------------------------------------------------------------------------- */
/* Certificates                                                               */
/* ------------------------------------------------------------------------- */

/* Cost of an explicit flux that carries a residual e (density, [ny][nx]).
 * This is an upper bound on the discrete W1 of the residual (it is not in the
 * paper; it turns f(m) into a certified upper bound when div m != rho).
 *
 * The flux is built on the dyadic tree of the grid: at each level every 2x2
 * block of current nodes sends its signed masses to the block's first node
 * along grid edges (offsets (1,0) and (0,1) cost one edge of the current
 * spacing, (1,1) costs two); the block's net mass then sits on that node and
 * the next level repeats with twice the spacing.  A dimension of extent 1 is
 * not pooled.  When a dimension is odd and larger than 1 the remaining nodes
 * route their positive mass to the negative mass along paths no longer than
 * the grid diameter D, costing at most D * max(positive mass, negative mass);
 * any imbalance (a residual that does not sum to zero, from rounding rho) is
 * charged D per unit of mass.  With p = 2 the same path flux costs no more,
 * since ||v||_2 <= ||v||_1 at every node. */
double w1o_route_bound(int nx, int ny, double h, const double* e)
{
    size_t n = (size_t)nx * (size_t)ny;
    double* q = (double*)malloc((n ? n : 1) * sizeof(double));
    if (!q) return NAN;
    for (size_t k = 0; k < n; ++k) q[k] = e[k] * h * h; /* masses */
    int cx = nx, cy = ny;
    double hx = h, hy = h, cost = 0.0;
    for (;;) {
        int px = (cx > 1 && cx % 2 == 0), py = (cy > 1 && cy % 2 == 0);
        int stop_x = (cx > 1 && cx % 2 == 1), stop_y = (cy > 1 && cy % 2 == 1);
        if (stop_x || stop_y || (!px && !py)) break;
        int bx = px ? 2 : 1, by = py ? 2 : 1;
        int ncx = cx / bx, ncy = cy / by;
        /* the current grid is stored with row stride nx inside q */
        for (int J = 0; J < ncy; ++J) {
            for (int I = 0; I < ncx; ++I) {
                double total = 0.0;
                for (int b = 0; b < by; ++b) {
                    for (int a = 0; a < bx; ++a) {
                        double qa = q[(size_t)(by * J + b) * (size_t)nx + (size_t)(bx * I + a)];
                        cost += fabs(qa) * (a * hx + b * hy);
                        total += qa;
                    }
                }
                q[(size_t)J * (size_t)nx + (size_t)I] = total;
            }
        }
        cx = ncx;
        cy = ncy;
        if (px) hx *= 2.0;
        if (py) hy *= 2.0;
    }
    double pos = 0.0, neg = 0.0;
    for (int J = 0; J < cy; ++J)
        for (int I = 0; I < cx; ++I) {
            double v = q[(size_t)J * (size_t)nx + (size_t)I];
            if (v > 0) pos += v; else neg -= v;
        }
    double diam = (cx - 1) * hx + (cy - 1) * hy;
    cost += diam * fmax(pos, neg);
    free(q);
    return cost;
}

/* Statistics of the state (m, phi) for the discrete problem with density rho.
 *
 * Dual sign: the Lagrangian of eq. minmax_cp is f(m) + <phi, A m - rho>_h, so
 * minimising over m gives the dual  max -<phi, rho>_h  s.t. ||grad phi(x)||_q <= 1
 * (eq. opt_dual3 up to the sign of phi, which the paper prints inconsistently).
 * phi / max(1, gmax) is dual feasible, so D(phi)/max(1, gmax) <= W1_h.
 * f(m) + route >= W1_h because m plus the residual flux is feasible. */
void w1o_stats(int nx, int ny, double h, int norm, const double* rho, const double* m1, const double* m2,
               const double* phi, w1o_stats_t* out)
{
    size_t n = (size_t)nx * (size_t)ny;
    double* d = (double*)calloc(n ? n : 1, sizeof(double));
    double* g1 = (double*)calloc(n ? n : 1, sizeof(double));
    double* g2 = (double*)calloc(n ? n : 1, sizeof(double));
    double* e = (double*)calloc(n ? n : 1, sizeof(double));
    memset(out, 0, sizeof(*out));
    if (!d || !g1 || !g2 || !e) {
        out->f = NAN;
        goto done;
    }
    w1o_div(nx, ny, h, m1, m2, d);
    w1o_grad(nx, ny, h, phi, g1, g2);
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            double a = AT(m1, j, i), b = AT(m2, j, i);
            if (i == nx - 1) a = 0.0; /* not a variable */
            if (j == ny - 1) b = 0.0;
            out->f += node_norm(norm, a, b) * h * h;
            out->dual -= AT(phi, j, i) * AT(rho, j, i) * h * h;
            AT(e, j, i) = AT(rho, j, i) - AT(d, j, i);
            out->res_l1 += fabs(AT(e, j, i)) * h * h;
            out->rho_l1 += fabs(AT(rho, j, i)) * h * h;
            double gq = node_dual_norm(norm, AT(g1, j, i), AT(g2, j, i));
            if (gq > out->gmax) out->gmax = gq;
        }
    }
    out->lb = out->dual / fmax(1.0, out->gmax);
    out->route = w1o_route_bound(nx, ny, h, e);
    out->ub = out->f + out->route;
    /* the saddle value: the min-max Lagrangian of eq. minmax_cp evaluated at
     * the state, L(m, phi) = f(m) + <phi, A_h m - rho>_h; at a saddle point it
     * equals W1_h, and near one it corrects f(m) for the residual A_h m - rho */
    {
        double inner = 0.0;
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) inner += AT(phi, j, i) * (AT(d, j, i) - AT(rho, j, i)) * h * h;
        out->saddle = out->f + inner;
    }
done:
    free(d); free(g1); free(g2); free(e);
}

/* ------------------------------------------------------------------------- */
/* Cross-level transfer (Sec. 3.2 and 3.3)                                    */
/* ------------------------------------------------------------------------- */

/* Coarse density on the level below: the mean of each 2x2 block, i.e. the
 * block's mass divided by the coarse cell area (Algorithm 3 passes rho to every
 * level without saying how it is coarsened; 2x2 sums of mass are the reading). */
void w1o_restrict(int nx, int ny, const double* fine, double* coarse)
{
    int ncx = nx / 2, ncy = ny / 2;
    for (int J = 0; J < ncy; ++J)
        for (int I = 0; I < ncx; ++I)
            coarse[(size_t)J * ncx + I] = 0.25 * (AT(fine, 2 * J, 2 * I) + AT(fine, 2 * J, 2 * I + 1) +
                                                  AT(fine, 2 * J + 1, 2 * I) + AT(fine, 2 * J + 1, 2 * I + 1));
}

/* Interpolate of Sec. 3.3 (eqs. inter_phi and inter_m) restated for pixel
 * grids nested by 2x2 agglomeration; coarse grid ncx x ncy, fine 2ncx x 2ncy.
 *
 * phi: each fine node averages the coarse nodes nearest to it, bilinearly: 3/4
 *   on its own coarse cell and 1/4 on the neighbouring coarse cell on its side,
 *   per axis (index clamped at the boundary).  Every coarse value keeps a total
 *   weight of 2 per axis, so Lemma 3.1 (non-expansiveness in L2) holds.
 * m1 along its own axis (nearest-neighbour rule of eq. inter_m): a fine x-edge
 *   that lies on a coarse x-edge (odd i) copies it; a fine x-edge inside a
 *   coarse cell (even i) takes the mean of the two coarse x-edges around that
 *   cell (the missing one at the left wall is 0).
 * m1 across its axis: both fine rows of a coarse row copy it (the paper
 *   averages across; copying keeps the restriction of div(Interpolate m) equal
 *   to the coarse div m, and every coarse value still has total weight 4).
 * m2 is the same with the axes exchanged. */
void w1o_prolong(int ncx, int ncy, const double* m1c, const double* m2c, const double* phic, double* m1f,
                 double* m2f, double* phif)
{
    const int nx = 2 * ncx, ny = 2 * ncy;
#define C(a, J, I) ((a)[(size_t)(J) * (size_t)ncx + (size_t)(I)])
    for (int j = 0; j < ny; ++j) {
        int J = j / 2;
        int Jn = (j % 2 == 0) ? J - 1 : J + 1;
        if (Jn < 0) Jn = 0;
        if (Jn > ncy - 1) Jn = ncy - 1;
        for (int i = 0; i < nx; ++i) {
            int I = i / 2;
            int In = (i % 2 == 0) ? I - 1 : I + 1;
            if (In < 0) In = 0;
            if (In > ncx - 1) In = ncx - 1;
            AT(phif, j, i) = 0.75 * 0.75 * C(phic, J, I) + 0.75 * 0.25 * C(phic, J, In) +
                             0.25 * 0.75 * C(phic, Jn, I) + 0.25 * 0.25 * C(phic, Jn, In);
            double v1;
            if (i % 2 == 1) {
                v1 = C(m1c, J, I);
            } else {
                double left = (I > 0) ? C(m1c, J, I - 1) : 0.0;
                v1 = 0.5 * (left + C(m1c, J, I));
            }
            if (i == nx - 1) v1 = 0.0;
            AT(m1f, j, i) = v1;
            double v2;
            if (j % 2 == 1) {
                v2 = C(m2c, J, I);
            } else {
                double below = (J > 0) ? C(m2c, J - 1, I) : 0.0;
                v2 = 0.5 * (below + C(m2c, J, I));
            }
            if (j == ny - 1) v2 = 0.0;
            AT(m2f, j, i) = v2;
        }
    }
#undef C
}

/* ------------------------------------------------------------------------- */
/* Algorithm 1 with a stopping test, and Algorithm 3                          */
/* ------------------------------------------------------------------------- */

/* Step sizes of eq. primaldual: mu = tau = theta / ||A_h|| with the Gershgorin
 * bound ||A_h|| <= 2 sqrt(d) / h, d = 2 (Sec. 4).  theta = 1/2 is the paper's
 * choice; theta = 1 is the faster choice of its footnote. */
double w1o_step_size(double h, double theta)
{
    return theta * h / (2.0 * sqrt(2.0));
}

static int converged(int stop_mode, const w1o_stats_t* st, double tol)
{
    if (stop_mode == W1O_STOP_FPR) return st->fpr < tol;
    if (st->ub <= 0.0) return 1; /* rho == 0 and m == 0: W1 = 0 */
    double lo = st->lb < st->f ? st->lb : st->f;
    return (st->ub - lo) <= tol * st->ub;
}

/* Algorithm 1 on one level, started from (m1, m2, phi), in place.
 * The stop test runs after every `check_every`-th step (k = K, 2K, ...), on the
 * step just taken (z^{k-1} -> z^k):
 *   fpr mode : R of eq. pd_stop for that step is below tol (the paper's rule;
 *              testing every K-th step instead of every step only delays the
 *              stop by less than K steps, since R^k is non-increasing);
 *   gap mode : (UB - min(LB, f)) <= tol * UB for z^k, i.e. f(m^k) is within a
 *              relative tol of the exact discrete W1_h (certified).
 * The level returns z^k.  If replay >= 0 the test is skipped and exactly
 * `replay` steps are taken.  Returns W1O_OK, or W1O_NOT_CONVERGED when
 * max_iters steps passed without the test passing. */
int w1o_solve_level(int nx, int ny, double h, int norm, double theta, double ratio, const double* rho, double* m1,
                    double* m2, double* phi, double tol, int stop_mode, int check_every, long max_iters, long replay,
                    long* iters_out, w1o_stats_t* stats_out)
{
    if (nx < 1 || ny < 1 || !(h > 0.0) || check_every < 1 || !(ratio > 0.0)) return W1O_ERR_ARG;
    /* mu tau = (theta / ||A_h||)^2 whatever the ratio tau / mu (the convergence
     * condition of eq. primaldual bounds the product only) */
    const double mu = w1o_step_size(h, theta) / sqrt(ratio), tau = w1o_step_size(h, theta) * sqrt(ratio);
    scratch_t s;
    if (scratch_alloc(&s, nx, ny) != W1O_OK) {
        scratch_free(&s);
        return W1O_ERR_NOMEM;
    }
    int status = W1O_NOT_CONVERGED;
    long k = 0;
    double last_fpr = 0.0;
    if (replay >= 0) {
        for (k = 0; k < replay; ++k) cp_step(&s, h, norm, mu, tau, rho, m1, m2, phi, NULL);
        status = W1O_OK;
    } else {
        for (;;) {
            const int check = ((k + 1) % check_every == 0);
            double fpr = 0.0;
            cp_step(&s, h, norm, mu, tau, rho, m1, m2, phi, check ? &fpr : NULL);
            ++k;
            if (!check) continue;
            last_fpr = fpr;
            int ok;
            if (stop_mode == W1O_STOP_FPR) {
                ok = fpr < tol;
            } else {
                w1o_stats_t st;
                w1o_stats(nx, ny, h, norm, rho, m1, m2, phi, &st);
                st.fpr = fpr;
                ok = converged(stop_mode, &st, tol);
            }
            if (ok) {
                status = W1O_OK;
                break;
            }
            if (k >= max_iters) break;
        }
    }
    if (iters_out) *iters_out = k;
    if (stats_out) {
        w1o_stats(nx, ny, h, norm, rho, m1, m2, phi, stats_out);
        stats_out->fpr = last_fpr;
    }
    scratch_free(&s);
    return status;
}

/* Algorithm 3: the cascadic multilevel version of Algorithm 1.
 *   - the finest density is rho = rho0 - rho1, checked for mass balance and
 *     made to sum to zero exactly (the constraint div m = rho has no solution
 *     otherwise, since the divergence of a zero-flux field sums to zero);
 *   - level l = levels is the finest grid nx x ny with spacing h; level l - 1
 *     has half the nodes per axis and twice the spacing (h_l = 2^{L-l} h);
 *   - coarse densities are 2x2 block means;
 *   - level 1 starts from m = 0, phi = 0; level l > 1 starts from Interpolate
 *     of level l - 1's result;
 *   - level l runs Algorithm 1 to tolerance tol_l = tol * (h_l / h)^alpha
 *     (eq. tol_formula_propose; alpha = -1 is the paper's recommendation).
 * replay (if not NULL) gives each level's exact iteration count.
 * Outputs: the finest (m1, m2, phi), the iterations per level, the stats of the
 * returned finest state, and *w1 = f(m) of the returned finest state. */
int w1o_multilevel(int nx, int ny, double h, int levels, int norm, double tol, double alpha, double theta,
                   double ratio, int stop_mode, int check_every, long max_iters, const double* rho0, const double* rho1,
                   const long* replay, double* m1_out, double* m2_out, double* phi_out, long* iters_out,
                   w1o_stats_t* stats_out, double* w1)
{
    if (nx < 1 || ny < 1 || levels < 1 || levels > 16 || check_every < 1) return W1O_ERR_ARG;
    if (!(h > 0.0)) h = 1.0 / (nx > ny ? nx : ny);
    const int div = 1 << (levels - 1);
    if (nx % div != 0 || ny % div != 0) return W1O_ERR_SHAPE;
    const size_t n = (size_t)nx * (size_t)ny;

    /* mass balance (the paper assumes two probability densities) */
    double M0 = 0.0, M1 = 0.0;
    for (size_t k = 0; k < n; ++k) {
        if (!isfinite(rho0[k]) || !isfinite(rho1[k])) return W1O_ERR_MASS;
        M0 += rho0[k] * h * h;
        M1 += rho1[k] * h * h;
    }
    if (fabs(M0 - M1) > 1e-6 * fmax(fabs(M0), fabs(M1))) return W1O_ERR_MASS;

    double** rho = (double**)calloc((size_t)levels, sizeof(double*));
    if (!rho) return W1O_ERR_NOMEM;
    int status = W1O_OK;
    for (int l = 0; l < levels; ++l) {
        size_t nl = (size_t)(nx >> (levels - 1 - l)) * (size_t)(ny >> (levels - 1 - l));
        rho[l] = (double*)calloc(nl, sizeof(double));
        if (!rho[l]) status = W1O_ERR_NOMEM;
    }
    double *m1 = NULL, *m2 = NULL, *phi = NULL, *c1 = NULL, *c2 = NULL, *cp = NULL;
    if (status != W1O_OK) goto out;

    /* finest rho = rho0 - rho1, shifted to sum exactly to zero */
    {
        double mean = 0.0;
        for (size_t k = 0; k < n; ++k) mean += rho0[k] - rho1[k];
        mean /= (double)n;
        for (size_t k = 0; k < n; ++k) rho[levels - 1][k] = (rho0[k] - rho1[k]) - mean;
    }
    for (int l = levels - 1; l > 0; --l) w1o_restrict(nx >> (levels - 1 - l), ny >> (levels - 1 - l), rho[l], rho[l - 1]);

    m1 = (double*)calloc(n, sizeof(double));
    m2 = (double*)calloc(n, sizeof(double));
    phi = (double*)calloc(n, sizeof(double));
    c1 = (double*)calloc(n, sizeof(double));
    c2 = (double*)calloc(n, sizeof(double));
    cp = (double*)calloc(n, sizeof(double));
    if (!m1 || !m2 || !phi || !c1 || !c2 || !cp) {
        status = W1O_ERR_NOMEM;
        goto out;
    }
    for (int l = 0; l < levels; ++l) {
        const int lnx = nx >> (levels - 1 - l), lny = ny >> (levels - 1 - l);
        const double hl = h * (double)(1 << (levels - 1 - l));
        if (l == 0) {
            memset(m1, 0, n * sizeof(double));
            memset(m2, 0, n * sizeof(double));
            memset(phi, 0, n * sizeof(double));
        } else {
            size_t nc = (size_t)(lnx / 2) * (size_t)(lny / 2);
            memcpy(c1, m1, nc * sizeof(double));
            memcpy(c2, m2, nc * sizeof(double));
            memcpy(cp, phi, nc * sizeof(double));
            w1o_prolong(lnx / 2, lny / 2, c1, c2, cp, m1, m2, phi);
        }
        const double tol_l = tol * pow(hl / h, alpha);
        long it = 0;
        w1o_stats_t st;
        int s = w1o_solve_level(lnx, lny, hl, norm, theta, ratio, rho[l], m1, m2, phi, tol_l, stop_mode, check_every,
                                max_iters, replay ? replay[l] : -1, &it, &st);
        if (iters_out) iters_out[l] = it;
        if (s < 0) {
            status = s;
            goto out;
        }
        if (s == W1O_NOT_CONVERGED) status = W1O_NOT_CONVERGED;
        if (l == levels - 1) {
            if (stats_out) *stats_out = st;
            if (w1) *w1 = st.f;
        }
    }
    memcpy(m1_out, m1, n * sizeof(double));
    memcpy(m2_out, m2, n * sizeof(double));
    memcpy(phi_out, phi, n * sizeof(double));
out:
    for (int l = 0; l < levels; ++l) free(rho[l]);
    free(rho);
    free(m1); free(m2); free(phi); free(c1); free(c2); free(cp);
    return status;
}

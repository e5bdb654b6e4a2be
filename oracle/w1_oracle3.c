/*
 * w1_oracle3.c -- FP64 CPU oracle of Algorithm 3 on three-dimensional grids.
 *
 * TEST INFRASTRUCTURE ONLY (see w1_oracle.c): the reference the CUDA 3-D path
 * is checked against.  The paper's setting is general d (Sec. 2.2, Sec. 4);
 * this file restates the d = 3 case on the pixel-centre (voxel-centre) grid:
 * nx x ny x nz nodes, spacing h, arrays [nz][ny][nx] (index (k ny + j) nx + i),
 * flux components m1 (x), m2 (y), m3 (z) with zero flux through the boundary
 * (m1[.][.][nx-1] = m2[.][ny-1][.] = m3[nz-1][.][.] = 0), inner products
 * weighted by h^3.  Plain loops in the paper's order, no blocking.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define AT3(a, k, j, i) (a)[((size_t)(k) * (size_t)ny + (size_t)(j)) * (size_t)nx + (size_t)(i)]

enum { N_L1 = 1, N_L2 = 2, N_LINF = 3 };

/* div^h: backward differences, pinned boundary flux ignored (zero). */
void w1o3_div(int nx, int ny, int nz, double h, const double* m1, const double* m2, const double* m3, double* out)
{
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double d1 = 0.0, d2 = 0.0, d3 = 0.0;
                if (i < nx - 1) d1 += AT3(m1, k, j, i);
                if (i > 0) d1 -= AT3(m1, k, j, i - 1);
                if (j < ny - 1) d2 += AT3(m2, k, j, i);
                if (j > 0) d2 -= AT3(m2, k, j - 1, i);
                if (k < nz - 1) d3 += AT3(m3, k, j, i);
                if (k > 0) d3 -= AT3(m3, k - 1, j, i);
                AT3(out, k, j, i) = d1 / h + d2 / h + d3 / h;
            }
}

/* Forward differences, zero where they would leave the grid (= -A_h^*). */
void w1o3_grad(int nx, int ny, int nz, double h, const double* phi, double* g1, double* g2, double* g3)
{
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                const double p = AT3(phi, k, j, i);
                AT3(g1, k, j, i) = (i < nx - 1) ? (AT3(phi, k, j, i + 1) - p) / h : 0.0;
                AT3(g2, k, j, i) = (j < ny - 1) ? (AT3(phi, k, j + 1, i) - p) / h : 0.0;
                AT3(g3, k, j, i) = (k < nz - 1) ? (AT3(phi, k + 1, j, i) - p) / h : 0.0;
            }
}

/* Euclidean projection of u onto the unit l1 ball in R^3 (sort the magnitudes,
 * find the shrink threshold). */
static void proj_l1_ball3(const double u[3], double p[3])
{
    double a[3] = {fabs(u[0]), fabs(u[1]), fabs(u[2])};
    if (a[0] + a[1] + a[2] <= 1.0) {
        p[0] = u[0];
        p[1] = u[1];
        p[2] = u[2];
        return;
    }
    double s[3] = {a[0], a[1], a[2]};
    for (int x = 0; x < 3; ++x) /* descending */
        for (int y = x + 1; y < 3; ++y)
            if (s[y] > s[x]) {
                double t = s[x];
                s[x] = s[y];
                s[y] = t;
            }
    double cum = 0.0, theta = 0.0;
    for (int r = 0; r < 3; ++r) {
        cum += s[r];
        double t = (cum - 1.0) / (double)(r + 1);
        if (s[r] - t > 0.0) theta = t;
    }
    for (int c = 0; c < 3; ++c) {
        double m = a[c] - theta;
        p[c] = m > 0.0 ? copysign(m, u[c]) : 0.0;
    }
}

/* Proximal map of mu ||.||_p at one node (the first line of eq. primaldual). */
static void prox3(int norm, double mu, const double v[3], double o[3])
{
    if (norm == N_L1) {
        for (int c = 0; c < 3; ++c) {
            double a = fabs(v[c]) - mu;
            o[c] = a > 0.0 ? copysign(a, v[c]) : 0.0;
        }
    } else if (norm == N_L2) {
        double n = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        double s = n > mu ? 1.0 - mu / n : 0.0;
        for (int c = 0; c < 3; ++c) o[c] = v[c] * s;
    } else {
        /* Moreau: prox_{mu ||.||_inf}(v) = v - mu Proj_{l1 ball}(v / mu) */
        double u[3] = {v[0] / mu, v[1] / mu, v[2] / mu}, p[3];
        proj_l1_ball3(u, p);
        for (int c = 0; c < 3; ++c) o[c] = v[c] - mu * p[c];
    }
}

void w1o3_prox(int norm, double mu, int n, const double* v1, const double* v2, const double* v3, double* o1,
               double* o2, double* o3)
{
    for (int k = 0; k < n; ++k) {
        double v[3] = {v1[k], v2[k], v3[k]}, o[3];
        prox3(norm, mu, v, o);
        o1[k] = o[0];
        o2[k] = o[1];
        o3[k] = o[2];
    }
}

static double node_norm3(int norm, double a, double b, double c)
{
    a = fabs(a);
    b = fabs(b);
    c = fabs(c);
    if (norm == N_L1) return a + b + c;
    if (norm == N_L2) return sqrt(a * a + b * b + c * c);
    return fmax(a, fmax(b, c));
}

static double node_dual_norm3(int norm, double a, double b, double c)
{
    return node_norm3(norm == N_L1 ? N_LINF : (norm == N_LINF ? N_L1 : N_L2), a, b, c);
}

/* mu = tau = theta / ||A_h|| with the Gershgorin bound ||A_h|| <= 2 sqrt(3) / h (d = 3). */
double w1o3_step_size(double h, double theta) { return theta * h / (2.0 * sqrt(3.0)); }

/* One step of eq. primaldual; fills fpr (if not NULL) with R^k of eq. pd_stop (h^3 weights). */
static int cp_step3(int nx, int ny, int nz, double h, int norm, double mu, double tau, const double* rho, double* m1,
                    double* m2, double* m3, double* phi, double* fpr)
{
    size_t n = (size_t)nx * ny * nz;
    double* w = (double*)malloc(9 * n * sizeof(double));
    if (!w) return -4;
    double *g1 = w, *g2 = w + n, *g3 = w + 2 * n, *b1 = w + 3 * n, *b2 = w + 4 * n, *b3 = w + 5 * n;
    double* d = w + 6 * n;
    double* dd = w + 7 * n;
    double* dp = w + 8 * n;
    w1o3_grad(nx, ny, nz, h, phi, g1, g2, g3);
    double sa = 0.0;
    for (size_t q = 0; q < n; ++q) {
        double v[3] = {m1[q] + mu * g1[q], m2[q] + mu * g2[q], m3[q] + mu * g3[q]}, o[3];
        prox3(norm, mu, v, o);
        size_t i = q % nx, j = (q / nx) % ny, k = q / ((size_t)nx * ny);
        if ((int)i == nx - 1) o[0] = 0.0;
        if ((int)j == ny - 1) o[1] = 0.0;
        if ((int)k == nz - 1) o[2] = 0.0;
        /* extrapolation mbar = 2 m' - m; keep dm = m' - m in g for the FPR */
        b1[q] = 2.0 * o[0] - m1[q];
        b2[q] = 2.0 * o[1] - m2[q];
        b3[q] = 2.0 * o[2] - m3[q];
        g1[q] = o[0] - m1[q];
        g2[q] = o[1] - m2[q];
        g3[q] = o[2] - m3[q];
        sa += g1[q] * g1[q] + g2[q] * g2[q] + g3[q] * g3[q];
        m1[q] = o[0];
        m2[q] = o[1];
        m3[q] = o[2];
    }
    w1o3_div(nx, ny, nz, h, b1, b2, b3, d);
    w1o3_div(nx, ny, nz, h, g1, g2, g3, dd);
    double sb = 0.0, sc = 0.0;
    for (size_t q = 0; q < n; ++q) {
        dp[q] = tau * (d[q] - rho[q]);
        phi[q] += dp[q];
        sb += dp[q] * dp[q];
        sc += dp[q] * dd[q];
    }
    if (fpr) *fpr = (sa / mu + sb / tau - 2.0 * sc) * h * h * h;
    free(w);
    return 0;
}

int w1o3_cp_iterate(int nx, int ny, int nz, double h, int norm, double mu, double tau, const double* rho, double* m1,
                    double* m2, double* m3, double* phi, long iters, double* fpr)
{
    double r = 0.0;
    for (long t = 0; t < iters; ++t) {
        int st = cp_step3(nx, ny, nz, h, norm, mu, tau, rho, m1, m2, m3, phi, &r);
        if (st) return st;
    }
    if (fpr) *fpr = r;
    return 0;
}

/* Certificates (the 3-D analogue of w1o_stats): f(m); LB = -<phi, rho>_h / max(1, max ||grad phi||_q);
 * UB = f(m) + cost of routing the residual along the dyadic octree. */
double w1o3_route_bound(int nx, int ny, int nz, double h, const double* e)
{
    size_t n = (size_t)nx * ny * nz;
    double* q = (double*)malloc((n ? n : 1) * sizeof(double));
    if (!q) return NAN;
    for (size_t t = 0; t < n; ++t) q[t] = e[t] * h * h * h;
    int cx = nx, cy = ny, cz = nz;
    double hx = h, hy = h, hz = h, cost = 0.0;
    for (;;) {
        int px = (cx > 1 && cx % 2 == 0), py = (cy > 1 && cy % 2 == 0), pz = (cz > 1 && cz % 2 == 0);
        int odd = (cx > 1 && cx % 2) || (cy > 1 && cy % 2) || (cz > 1 && cz % 2);
        if (odd || (!px && !py && !pz)) break;
        int bx = px ? 2 : 1, by = py ? 2 : 1, bz = pz ? 2 : 1;
        int ncx = cx / bx, ncy = cy / by, ncz = cz / bz;
        for (int K = 0; K < ncz; ++K)
            for (int J = 0; J < ncy; ++J)
                for (int I = 0; I < ncx; ++I) {
                    double total = 0.0;
                    for (int c = 0; c < bz; ++c)
                        for (int b = 0; b < by; ++b)
                            for (int a = 0; a < bx; ++a) {
                                double qa = AT3(q, bz * K + c, by * J + b, bx * I + a);
                                cost += fabs(qa) * (a * hx + b * hy + c * hz);
                                total += qa;
                            }
                    AT3(q, K, J, I) = total;
                }
        cx = ncx;
        cy = ncy;
        cz = ncz;
        if (px) hx *= 2.0;
        if (py) hy *= 2.0;
        if (pz) hz *= 2.0;
    }
    double pos = 0.0, neg = 0.0;
    for (int K = 0; K < cz; ++K)
        for (int J = 0; J < cy; ++J)
            for (int I = 0; I < cx; ++I) {
                double v = AT3(q, K, J, I);
                if (v > 0) pos += v;
                else neg -= v;
            }
    cost += ((cx - 1) * hx + (cy - 1) * hy + (cz - 1) * hz) * fmax(pos, neg);
    free(q);
    return cost;
}

typedef struct {
    double f, dual, res_l1, rho_l1, gmax, lb, route, ub;
    double saddle; /* L(m, phi) = f(m) + <phi, A m - rho>_h, the Lagrangian of eq. minmax_cp */
} w1o3_stats_t;

void w1o3_stats(int nx, int ny, int nz, double h, int norm, const double* rho, const double* m1, const double* m2,
                const double* m3, const double* phi, w1o3_stats_t* out)
{
    size_t n = (size_t)nx * ny * nz;
    double h3 = h * h * h;
    double* w = (double*)malloc(5 * n * sizeof(double));
    memset(out, 0, sizeof(*out));
    if (!w) return;
    double *d = w, *g1 = w + n, *g2 = w + 2 * n, *g3 = w + 3 * n, *e = w + 4 * n;
    w1o3_div(nx, ny, nz, h, m1, m2, m3, d);
    w1o3_grad(nx, ny, nz, h, phi, g1, g2, g3);
    double f = 0.0, dual = 0.0, res = 0.0, rl = 0.0, gmax = 0.0;
    for (size_t q = 0; q < n; ++q) {
        f += node_norm3(norm, m1[q], m2[q], m3[q]);
        dual -= phi[q] * rho[q];
        e[q] = rho[q] - d[q];
        res += fabs(e[q]);
        rl += fabs(rho[q]);
        gmax = fmax(gmax, node_dual_norm3(norm, g1[q], g2[q], g3[q]));
    }
    out->f = f * h3;
    out->dual = dual * h3;
    out->res_l1 = res * h3;
    out->rho_l1 = rl * h3;
    out->gmax = gmax;
    out->lb = out->dual / fmax(1.0, gmax);
    out->route = w1o3_route_bound(nx, ny, nz, h, e);
    out->ub = out->f + out->route;
    double inner = 0.0; /* <phi, A m - rho>_h */
    for (size_t q = 0; q < n; ++q) inner += phi[q] * (d[q] - rho[q]) * h3;
    out->saddle = out->f + inner;
    free(w);
}

/* Coarse density: mean of each 2x2x2 block (Algorithm 3's rho on level l - 1). */
void w1o3_restrict(int nx, int ny, int nz, const double* fine, double* coarse)
{
    int ncx = nx / 2, ncy = ny / 2, ncz = nz / 2;
    for (int K = 0; K < ncz; ++K)
        for (int J = 0; J < ncy; ++J)
            for (int I = 0; I < ncx; ++I) {
                double s = 0.0;
                for (int c = 0; c < 2; ++c)
                    for (int b = 0; b < 2; ++b)
                        for (int a = 0; a < 2; ++a) s += AT3(fine, 2 * K + c, 2 * J + b, 2 * I + a);
                coarse[((size_t)K * ncy + J) * ncx + I] = s / 8.0;
            }
}

/* Interpolate of Sec. 3.3 restated on voxel centres: phi trilinear (3/4 own cell,
 * 1/4 the neighbour on the fine node's side, per axis, clamped); each flux
 * component along its own axis copies the coarse edge on odd fine edges and
 * averages the two coarse edges of the cell on even ones, and copies across the
 * other two axes. */
void w1o3_prolong(int ncx, int ncy, int ncz, const double* m1c, const double* m2c, const double* m3c,
                  const double* phic, double* m1f, double* m2f, double* m3f, double* phif)
{
    int nx = 2 * ncx, ny = 2 * ncy, nz = 2 * ncz;
#define C3(a, K, J, I) (a)[((size_t)(K) * (size_t)ncy + (size_t)(J)) * (size_t)ncx + (size_t)(I)]
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                int I = i / 2, J = j / 2, K = k / 2;
                int In = (i % 2) ? I + 1 : I - 1, Jn = (j % 2) ? J + 1 : J - 1, Kn = (k % 2) ? K + 1 : K - 1;
                if (In < 0) In = 0;
                if (In > ncx - 1) In = ncx - 1;
                if (Jn < 0) Jn = 0;
                if (Jn > ncy - 1) Jn = ncy - 1;
                if (Kn < 0) Kn = 0;
                if (Kn > ncz - 1) Kn = ncz - 1;
                double p = 0.0;
                for (int c = 0; c < 2; ++c)
                    for (int b = 0; b < 2; ++b)
                        for (int a = 0; a < 2; ++a) {
                            double w = (a ? 0.25 : 0.75) * (b ? 0.25 : 0.75) * (c ? 0.25 : 0.75);
                            p += w * C3(phic, c ? Kn : K, b ? Jn : J, a ? In : I);
                        }
                AT3(phif, k, j, i) = p;
                double v1, v2, v3;
                if (i % 2) v1 = C3(m1c, K, J, I);
                else v1 = 0.5 * ((I > 0 ? C3(m1c, K, J, I - 1) : 0.0) + C3(m1c, K, J, I));
                if (j % 2) v2 = C3(m2c, K, J, I);
                else v2 = 0.5 * ((J > 0 ? C3(m2c, K, J - 1, I) : 0.0) + C3(m2c, K, J, I));
                if (k % 2) v3 = C3(m3c, K, J, I);
                else v3 = 0.5 * ((K > 0 ? C3(m3c, K - 1, J, I) : 0.0) + C3(m3c, K, J, I));
                AT3(m1f, k, j, i) = i == nx - 1 ? 0.0 : v1;
                AT3(m2f, k, j, i) = j == ny - 1 ? 0.0 : v2;
                AT3(m3f, k, j, i) = k == nz - 1 ? 0.0 : v3;
            }
#undef C3
}

/* Algorithm 1 on one 3-D grid with the FPR stop (R^k < tol tested after every
 * K-th step) or exactly `replay` steps; returns 0 converged, 1 cap reached. */
int w1o3_solve_level(int nx, int ny, int nz, double h, int norm, double theta, const double* rho, double* m1,
                     double* m2, double* m3, double* phi, double tol, int check_every, long max_iters, long replay,
                     long* iters, double* fpr_out)
{
    double mu = w1o3_step_size(h, theta), r = 0.0;
    long k = 0;
    for (;;) {
        if (replay >= 0 && k >= replay) break;
        if (replay < 0 && k >= max_iters) {
            *iters = k;
            *fpr_out = r;
            return 1;
        }
        int st = cp_step3(nx, ny, nz, h, norm, mu, mu, rho, m1, m2, m3, phi, &r);
        if (st) return st;
        ++k;
        if (replay < 0 && k % check_every == 0 && r < tol) break;
    }
    *iters = k;
    *fpr_out = r;
    return 0;
}

/* Algorithm 3 on 3-D grids: restriction pyramid, coarse to fine, each level
 * started from the interpolated coarser solution (zero on the coarsest),
 * eps_l = tol (h_l / h)^alpha.  Mass check and exact zero mean as in 2-D.
 * Returns 0, 1 (a level hit max_iters), or -1 / -2 / -3 / -4 (argument, shape,
 * mass, memory). */
int w1o3_multilevel(int nx, int ny, int nz, double h, int levels, int norm, double tol, double alpha, double theta,
                    int check_every, long max_iters, const double* rho0, const double* rho1, const long* replay,
                    double* m1, double* m2, double* m3, double* phi, long* iters, double* fprs, w1o3_stats_t* stats,
                    double* w1)
{
    if (nx < 1 || ny < 1 || nz < 1 || levels < 1 || levels > 16 || check_every < 1) return -1;
    if (h <= 0.0) h = 1.0 / fmax(nx, fmax(ny, nz));
    int div = 1 << (levels - 1);
    if (nx % div || ny % div || nz % div) return -2;
    size_t n = (size_t)nx * ny * nz;
    double M0 = 0.0, M1 = 0.0, h3 = h * h * h;
    for (size_t q = 0; q < n; ++q) {
        if (!isfinite(rho0[q]) || !isfinite(rho1[q])) return -3;
        M0 += rho0[q] * h3;
        M1 += rho1[q] * h3;
    }
    if (fabs(M0 - M1) > 1e-6 * fmax(fabs(M0), fabs(M1))) return -3;
    double** pyr = (double**)calloc((size_t)levels, sizeof(double*));
    double* state = (double*)malloc(8 * n * sizeof(double)); /* two sets of m1 m2 m3 phi */
    if (!pyr || !state) {
        free(pyr);
        free(state);
        return -4;
    }
    int ret = 0;
    pyr[levels - 1] = (double*)malloc(n * sizeof(double));
    if (!pyr[levels - 1]) ret = -4;
    double mean = 0.0;
    for (size_t q = 0; q < n && !ret; ++q) mean += rho0[q] - rho1[q];
    mean /= (double)n;
    for (size_t q = 0; q < n && !ret; ++q) pyr[levels - 1][q] = (rho0[q] - rho1[q]) - mean;
    for (int l = levels - 1; l > 0 && !ret; --l) {
        int sh = levels - 1 - l;
        int fx = nx >> sh, fy = ny >> sh, fz = nz >> sh;
        pyr[l - 1] = (double*)malloc((size_t)(fx / 2) * (fy / 2) * (fz / 2) * sizeof(double));
        if (!pyr[l - 1]) ret = -4;
        else w1o3_restrict(fx, fy, fz, pyr[l], pyr[l - 1]);
    }
    double* cur = state;
    double* prev = state + 4 * n;
    for (int l = 0; l < levels && ret >= 0 && ret != -4; ++l) {
        int sh = levels - 1 - l;
        int lx = nx >> sh, ly = ny >> sh, lz = nz >> sh;
        size_t ln = (size_t)lx * ly * lz;
        double hl = h * (double)(1 << sh);
        double *c1 = cur, *c2 = cur + ln, *c3 = cur + 2 * ln, *cp = cur + 3 * ln;
        if (l == 0) {
            memset(cur, 0, 4 * ln * sizeof(double));
        } else {
            size_t pn = (size_t)(lx / 2) * (ly / 2) * (lz / 2);
            w1o3_prolong(lx / 2, ly / 2, lz / 2, prev, prev + pn, prev + 2 * pn, prev + 3 * pn, c1, c2, c3, cp);
        }
        double tl = tol * pow(hl / h, alpha);
        int st = w1o3_solve_level(lx, ly, lz, hl, norm, theta, pyr[l], c1, c2, c3, cp, tl, check_every, max_iters,
                                  replay ? replay[l] : -1, &iters[l], &fprs[l]);
        if (st < 0) ret = st;
        else if (st == 1) ret = 1;
        double* t = cur;
        cur = prev;
        prev = t;
    }
    if (ret >= 0) {
        /* the finest state is in prev */
        memcpy(m1, prev, n * sizeof(double));
        memcpy(m2, prev + n, n * sizeof(double));
        memcpy(m3, prev + 2 * n, n * sizeof(double));
        memcpy(phi, prev + 3 * n, n * sizeof(double));
        w1o3_stats(nx, ny, nz, h, norm, pyr[levels - 1], m1, m2, m3, phi, stats);
        *w1 = stats->f;
    }
    for (int l = 0; l < levels; ++l) free(pyr[l]);
    free(pyr);
    free(state);
    return ret;
}

/*
 * Plain FP64 CPU oracle of the parametric lattice Boltzmann method (PLBM).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * restatement of the method that the CUDA path is checked against.  Only the
 * test suite, the smoke check and the CPU-baseline leg of the benchmark may
 * load it.  It shares no code, header or constant table with the CUDA path.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (oracle/__init__.py, build()).
 * -ffp-contract=off keeps every product and sum rounded separately, so the
 * result only depends on the order of operations written below.
 *
 * Paper: J. W. Shim, "Parametric Lattice Boltzmann Method" (arXiv:1402.5487).
 *   Eq. (eq:density)/(eq:eqdist): f_i = rho p_i, f^eq_i = rho r_i.
 *   Eq. (eq:srt): f_i(x + v_i dt, t + dt) = (1 - omega) f_i(x,t) + omega f^eq_i(x,t).
 *   Eq. (eq:rdr): r_i = sum_j c_ij mu_{j-1}; c_ij is the coefficient of degree
 *   j-1 of the Lagrange polynomial through (v_k, delta_ik); mu_n = int v^n F dv.
 *   Appendix, Eq. (eq:constraints): R = V^{-1} M with V_{n,k} = v_k^n.
 *   Sec. 2.1: multi-dimensional models are tensor products of 1D models.
 *
 * Readings taken where the paper is silent (all lattice units, dx = dt = 1):
 *   - Eq. (eq:srt) is a push; the oracle stores the post-collision state and
 *     advances by "pull then collide", which gives the same sequence of
 *     post-collision states.
 *   - rho = sum f, rho u = sum v f, d rho theta = sum |v - u|^2 f (d = dim),
 *     consistent with the (d/2) rho theta energy of Eq. (eq:ns).
 *   - 2D uses one scalar theta for both tensor factors (isotropic Maxwellian
 *     of the Appendix).
 *   - Fixed ends ("the extreme left and right are maintained by C_L and C_R",
 *     Sec. 3.2): nodes left of x = 0 and right of x = nx-1 hold f^eq(C_L) and
 *     f^eq(C_R) for ever.
 *   - Isothermal models (Eq. eq:1d3v, Table 1) are the general rule with theta
 *     held at theta_0 in the equilibrium.
 *
 * Population index in 2D: p = ix * q1 + iy, velocity (v[ix], v[iy]).
 * Array layout: f[p][y][x], x fastest, no padding.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXQ1 8
#define ORC_MAXQ (ORC_MAXQ1 * ORC_MAXQ1)

typedef struct {
    int dim;          /* 1 or 2 */
    int q1;           /* velocities per axis */
    int nx, ny;       /* ny = 1 in 1D */
    int bc;           /* 0 periodic; 1 fixed ends in x (y periodic in 2D) */
    int isothermal;   /* 1: theta in the equilibrium is held at theta0 */
    int v[ORC_MAXQ1];
    double omega;
    double theta0;
    double C[ORC_MAXQ1 * ORC_MAXQ1];   /* C[i*q1 + n]: coefficient of v^n in L_i */
    double ghost_left[ORC_MAXQ];       /* f^eq(C_L) for fixed ends */
    double ghost_right[ORC_MAXQ];      /* f^eq(C_R) for fixed ends */
} orc_lattice;

int orc_sizeof_lattice(void) { return (int)sizeof(orc_lattice); }

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Appendix, Eq. (eq:constraints) with n* = q-1: R = V^{-1} M, V_{n,k} = v_k^n.
 * C = V^{-1} by Gauss-Jordan elimination with partial pivoting on [V | I].
 * Row i of C holds the monomial coefficients of the Lagrange polynomial L_i
 * (Eq. eq:rdr): sum_n C[i][n] v_k^n = delta_ik.
 * Returns 0 on success, -1 if V is singular (repeated velocities).
 */
int orc_vandermonde_inverse(int q, const double *v, double *C)
{
    double A[ORC_MAXQ1][2 * ORC_MAXQ1];
    if (q < 1 || q > ORC_MAXQ1) return -1;
    for (int n = 0; n < q; ++n) {
        for (int k = 0; k < q; ++k) {
            double p = 1.0;
            for (int e = 0; e < n; ++e) p = p * v[k];
            A[n][k] = p;
            A[n][q + k] = (n == k) ? 1.0 : 0.0;
        }
    }
    for (int col = 0; col < q; ++col) {
        int piv = col;
        for (int r = col + 1; r < q; ++r)
            if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
        if (A[piv][col] == 0.0) return -1;
        if (piv != col) {
            for (int c = 0; c < 2 * q; ++c) {
                double t = A[col][c];
                A[col][c] = A[piv][c];
                A[piv][c] = t;
            }
        }
        double d = A[col][col];
        for (int c = 0; c < 2 * q; ++c) A[col][c] = A[col][c] / d;
        for (int r = 0; r < q; ++r) {
            if (r == col) continue;
            double m = A[r][col];
            if (m == 0.0) continue;
            for (int c = 0; c < 2 * q; ++c) A[r][c] = A[r][c] - m * A[col][c];
        }
    }
    /* [V | I] -> [I | V^{-1}];  C = V^{-1}, C[i][n] multiplies mu_n. */
    for (int i = 0; i < q; ++i)
        for (int n = 0; n < q; ++n) C[i * q + n] = A[i][q + n];
    return 0;
}

/*
 * Raw moments of the 1D Maxwell-Boltzmann (Gaussian) distribution with mean u
 * and variance theta, mu_n = int v^n F(v) dv (Eq. eq:rdr, Appendix):
 * mu_0 = 1, mu_1 = u, mu_{n+1} = u mu_n + n theta mu_{n-1}.
 * This recurrence reproduces the Maxwell-Boltzmann row of Table 2.
 */
void orc_mb_moments(double u, double theta, int nmax, double *mu)
{
    mu[0] = 1.0;
    if (nmax >= 1) mu[1] = u;
    for (int n = 1; n < nmax; ++n) mu[n + 1] = u * mu[n] + n * theta * mu[n - 1];
}

/* Eq. (eq:rdr): r_i = sum_{j=1}^{q} c_ij mu_{j-1}. */
void orc_r1d(int q1, const double *C, double u, double theta, double *r)
{
    double mu[ORC_MAXQ1];
    orc_mb_moments(u, theta, q1 - 1, mu);
    for (int i = 0; i < q1; ++i) {
        double s = 0.0;
        for (int n = 0; n < q1; ++n) s = s + C[i * q1 + n] * mu[n];
        r[i] = s;
    }
}

/*
 * Eq. (eq:eqdist) with the tensor-product rule of Sec. 2.1:
 * 1D: f^eq_i = rho r_i(u, theta);
 * 2D: f^eq_{(ix,iy)} = rho r_ix(u_x, theta) r_iy(u_y, theta).
 */
void orc_feq(int dim, int q1, const double *C, double rho, double ux, double uy,
             double theta, double *feq)
{
    double rx[ORC_MAXQ1], ry[ORC_MAXQ1];
    orc_r1d(q1, C, ux, theta, rx);
    if (dim == 1) {
        for (int i = 0; i < q1; ++i) feq[i] = rho * rx[i];
        return;
    }
    orc_r1d(q1, C, uy, theta, ry);
    for (int ix = 0; ix < q1; ++ix)
        for (int iy = 0; iy < q1; ++iy) feq[ix * q1 + iy] = rho * rx[ix] * ry[iy];
}

/*
 * Macroscopic fields of one node from its populations:
 * rho = sum f, rho u = sum v f, d rho theta = sum |v|^2 f - rho |u|^2.
 */
void orc_node_moments(const orc_lattice *L, const double *f, double *rho_o,
                      double *ux_o, double *uy_o, double *theta_o)
{
    int q = (L->dim == 1) ? L->q1 : L->q1 * L->q1;
    double rho = 0.0, jx = 0.0, jy = 0.0, e = 0.0;
    for (int p = 0; p < q; ++p) {
        int ix = (L->dim == 1) ? p : p / L->q1;
        int iy = (L->dim == 1) ? 0 : p % L->q1;
        double vx = L->v[ix];
        double vy = (L->dim == 1) ? 0.0 : (double)L->v[iy];
        rho = rho + f[p];
        jx = jx + vx * f[p];
        jy = jy + vy * f[p];
        e = e + (vx * vx + vy * vy) * f[p];
    }
    double ux = jx / rho;
    double uy = jy / rho;
    double theta = (e / rho - (ux * ux + uy * uy)) / L->dim;
    *rho_o = rho;
    *ux_o = ux;
    *uy_o = uy;
    *theta_o = theta;
}

/*
 * BGK collision of one node, Eq. (eq:srt) right-hand side:
 * f_out = (1 - omega) f_in + omega f^eq(rho, u, theta of f_in).
 */
void orc_collide_node(const orc_lattice *L, const double *fin, double *fout)
{
    int q = (L->dim == 1) ? L->q1 : L->q1 * L->q1;
    double rho, ux, uy, theta, feq[ORC_MAXQ];
    orc_node_moments(L, fin, &rho, &ux, &uy, &theta);
    if (L->isothermal) theta = L->theta0;
    orc_feq(L->dim, L->q1, L->C, rho, ux, uy, theta, feq);
    for (int p = 0; p < q; ++p)
        fout[p] = (1.0 - L->omega) * fin[p] + L->omega * feq[p];
}

/*
 * One time step, Eq. (eq:srt) read as pull + collide on post-collision states:
 * f_in,p(x) = f_p(x - v_p) (periodic wrap, or a frozen ghost population for
 * fixed ends), then f_dst,p(x) = (1 - omega) f_in,p + omega f^eq_p.
 */
void orc_step(const orc_lattice *L, const double *fsrc, double *fdst)
{
    const int nx = L->nx, ny = L->ny, q1 = L->q1;
    const int q = (L->dim == 1) ? q1 : q1 * q1;
    const long plane = (long)nx * ny;
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
    for (int y = 0; y < ny; ++y) {
        double fin[ORC_MAXQ], fout[ORC_MAXQ];
        for (int x = 0; x < nx; ++x) {
            for (int p = 0; p < q; ++p) {
                int ix = (L->dim == 1) ? p : p / q1;
                int iy = (L->dim == 1) ? 0 : p % q1;
                int sx = x - L->v[ix];
                int sy = (L->dim == 1) ? 0 : y - L->v[iy];
                sy = ((sy % ny) + ny) % ny;
                if (L->bc == 1) {
                    if (sx < 0) { fin[p] = L->ghost_left[p]; continue; }
                    if (sx >= nx) { fin[p] = L->ghost_right[p]; continue; }
                } else {
                    sx = ((sx % nx) + nx) % nx;
                }
                fin[p] = fsrc[p * plane + (long)sy * nx + sx];
            }
            orc_collide_node(L, fin, fout);
            for (int p = 0; p < q; ++p) fdst[p * plane + (long)y * nx + x] = fout[p];
        }
    }
}

/* n steps alternating between buffers a and b; the final state is left in a. */
void orc_run(const orc_lattice *L, double *a, double *b, long nsteps)
{
    const int q = (L->dim == 1) ? L->q1 : L->q1 * L->q1;
    const long total = (long)q * L->nx * L->ny;
    double *src = a, *dst = b;
    for (long s = 0; s < nsteps; ++s) {
        orc_step(L, src, dst);
        double *t = src;
        src = dst;
        dst = t;
    }
    if (src != a) memcpy(a, src, sizeof(double) * (size_t)total);
}

/* Initial state: f = f^eq(rho, u, theta) at every node (a post-collision state). */
void orc_init(const orc_lattice *L, const double *rho, const double *ux, const double *uy,
              const double *theta, double *f)
{
    const int q = (L->dim == 1) ? L->q1 : L->q1 * L->q1;
    const long plane = (long)L->nx * L->ny;
    for (long n = 0; n < plane; ++n) {
        double feq[ORC_MAXQ];
        double th = L->isothermal ? L->theta0 : theta[n];
        orc_feq(L->dim, L->q1, L->C, rho[n], ux[n], (L->dim == 1) ? 0.0 : uy[n], th, feq);
        for (int p = 0; p < q; ++p) f[p * plane + n] = feq[p];
    }
}

/* Fields rho, u_x, u_y, theta of every node of a stored population array. */
void orc_moments(const orc_lattice *L, const double *f, double *rho, double *ux,
                 double *uy, double *theta)
{
    const int q = (L->dim == 1) ? L->q1 : L->q1 * L->q1;
    const long plane = (long)L->nx * L->ny;
    for (long n = 0; n < plane; ++n) {
        double fn[ORC_MAXQ], r, a, b, t;
        for (int p = 0; p < q; ++p) fn[p] = f[p * plane + n];
        orc_node_moments(L, fn, &r, &a, &b, &t);
        rho[n] = r;
        ux[n] = a;
        if (uy) uy[n] = b;
        theta[n] = t;
    }
}

/* Neumaier compensated sum step. */
static void neu_add(double *s, double *c, double x)
{
    double t = *s + x;
    if (fabs(*s) >= fabs(x)) *c = *c + ((*s - t) + x);
    else *c = *c + ((x - t) + *s);
    *s = t;
}

/*
 * Global conserved sums over all nodes: out[0] mass sum f, out[1..2] momentum
 * sum v f, out[3] energy sum |v|^2 f.  Compensated summation in FP64.
 */
void orc_conserved(const orc_lattice *L, const double *f, double *out)
{
    const int q = (L->dim == 1) ? L->q1 : L->q1 * L->q1;
    const long plane = (long)L->nx * L->ny;
    double s[4] = {0, 0, 0, 0}, c[4] = {0, 0, 0, 0};
    for (int p = 0; p < q; ++p) {
        int ix = (L->dim == 1) ? p : p / L->q1;
        int iy = (L->dim == 1) ? 0 : p % L->q1;
        double vx = L->v[ix];
        double vy = (L->dim == 1) ? 0.0 : (double)L->v[iy];
        for (long n = 0; n < plane; ++n) {
            double fv = f[p * plane + n];
            neu_add(&s[0], &c[0], fv);
            neu_add(&s[1], &c[1], vx * fv);
            neu_add(&s[2], &c[2], vy * fv);
            neu_add(&s[3], &c[3], (vx * vx + vy * vy) * fv);
        }
    }
    for (int k = 0; k < 4; ++k) out[k] = s[k] + c[k];
}

/* ======================================================================
 * Three dimensions (Sec. 2.1: the D3 models are the tensor product of three
 * 1D rules with one scalar theta).  A separate description and separate
 * functions keep the 1D/2D code above unchanged.
 *
 * Population index: p = (ix * q1 + iy) * q1 + iz, velocity (v[ix], v[iy], v[iz]).
 * Array layout: f[p][z][y][x], x fastest, no padding.  Periodic in x, y and z.
 * theta = (sum |v|^2 f / rho - |u|^2) / 3.
 * ====================================================================== */
#define ORC3_MAXQ1 5
#define ORC3_MAXQ (ORC3_MAXQ1 * ORC3_MAXQ1 * ORC3_MAXQ1)

typedef struct {
    int q1;
    int nx, ny, nz;
    int isothermal;
    int v[ORC3_MAXQ1];
    double omega;
    double theta0;
    double C[ORC3_MAXQ1 * ORC3_MAXQ1];
} orc_lattice3;

int orc3_sizeof_lattice(void) { return (int)sizeof(orc_lattice3); }

/* f^eq_{(ix,iy,iz)} = rho r_ix(u_x) r_iy(u_y) r_iz(u_z), one theta for the three factors. */
void orc3_feq(int q1, const double *C, double rho, double ux, double uy, double uz,
              double theta, double *feq)
{
    double ra[ORC3_MAXQ1], rb[ORC3_MAXQ1], rc[ORC3_MAXQ1];
    orc_r1d(q1, C, ux, theta, ra);
    orc_r1d(q1, C, uy, theta, rb);
    orc_r1d(q1, C, uz, theta, rc);
    for (int a = 0; a < q1; ++a)
        for (int b = 0; b < q1; ++b)
            for (int c = 0; c < q1; ++c) feq[(a * q1 + b) * q1 + c] = rho * ra[a] * rb[b] * rc[c];
}

/* rho = sum f; rho u = sum v f; 3 rho theta = sum |v|^2 f - rho |u|^2. */
void orc3_node_moments(const orc_lattice3 *L, const double *f, double *m_out)
{
    const int q1 = L->q1;
    double m0 = 0.0, mx = 0.0, my = 0.0, mz = 0.0, en = 0.0;
    for (int a = 0; a < q1; ++a)
        for (int b = 0; b < q1; ++b)
            for (int c = 0; c < q1; ++c) {
                const double fv = f[(a * q1 + b) * q1 + c];
                const double cx = L->v[a], cy = L->v[b], cz = L->v[c];
                m0 = m0 + fv;
                mx = mx + cx * fv;
                my = my + cy * fv;
                mz = mz + cz * fv;
                en = en + (cx * cx + cy * cy + cz * cz) * fv;
            }
    const double wx = mx / m0, wy = my / m0, wz = mz / m0;
    m_out[0] = m0;
    m_out[1] = wx;
    m_out[2] = wy;
    m_out[3] = wz;
    m_out[4] = (en / m0 - (wx * wx + wy * wy + wz * wz)) / 3.0;
}

/* BGK collision of one node: fo = (1 - omega) fi + omega f^eq(moments of fi). */
void orc3_collide_node(const orc_lattice3 *L, const double *fi, double *fo)
{
    const int q = L->q1 * L->q1 * L->q1;
    double m[5], fe[ORC3_MAXQ];
    orc3_node_moments(L, fi, m);
    const double th = L->isothermal ? L->theta0 : m[4];
    orc3_feq(L->q1, L->C, m[0], m[1], m[2], m[3], th, fe);
    for (int p = 0; p < q; ++p) fo[p] = (1.0 - L->omega) * fi[p] + L->omega * fe[p];
}

static int orc3_wrap(int i, int n) { return ((i % n) + n) % n; }

/* One step: pull f_p(x - v_p) with periodic wrap in x, y, z, then collide. */
void orc3_step(const orc_lattice3 *L, const double *fsrc, double *fdst)
{
    const int nx = L->nx, ny = L->ny, nz = L->nz, q1 = L->q1;
    const long vol = (long)nx * ny * nz;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) collapse(2)
#endif
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y) {
            double fi[ORC3_MAXQ], fo[ORC3_MAXQ];
            for (int x = 0; x < nx; ++x) {
                for (int a = 0; a < q1; ++a)
                    for (int b = 0; b < q1; ++b)
                        for (int c = 0; c < q1; ++c) {
                            const int p = (a * q1 + b) * q1 + c;
                            const int px = orc3_wrap(x - L->v[a], nx);
                            const int py = orc3_wrap(y - L->v[b], ny);
                            const int pz = orc3_wrap(z - L->v[c], nz);
                            fi[p] = fsrc[p * vol + ((long)pz * ny + py) * nx + px];
                        }
                orc3_collide_node(L, fi, fo);
                const int q = q1 * q1 * q1;
                for (int p = 0; p < q; ++p) fdst[p * vol + ((long)z * ny + y) * nx + x] = fo[p];
            }
        }
}

void orc3_run(const orc_lattice3 *L, double *a, double *b, long nsteps)
{
    const long total = (long)L->q1 * L->q1 * L->q1 * L->nx * L->ny * L->nz;
    double *src = a, *dst = b;
    for (long s = 0; s < nsteps; ++s) {
        orc3_step(L, src, dst);
        double *t = src;
        src = dst;
        dst = t;
    }
    if (src != a) memcpy(a, src, sizeof(double) * (size_t)total);
}

/* f = f^eq(rho, u, theta) at every node; fields are [z][y][x]. */
void orc3_init(const orc_lattice3 *L, const double *rho, const double *ux, const double *uy,
               const double *uz, const double *theta, double *f)
{
    const int q = L->q1 * L->q1 * L->q1;
    const long vol = (long)L->nx * L->ny * L->nz;
    for (long n = 0; n < vol; ++n) {
        double fe[ORC3_MAXQ];
        const double th = L->isothermal ? L->theta0 : theta[n];
        orc3_feq(L->q1, L->C, rho[n], ux[n], uy[n], uz[n], th, fe);
        for (int p = 0; p < q; ++p) f[p * vol + n] = fe[p];
    }
}

/* Fields of every node: out[k * vol + n], k = rho, u_x, u_y, u_z, theta. */
void orc3_moments(const orc_lattice3 *L, const double *f, double *out)
{
    const int q = L->q1 * L->q1 * L->q1;
    const long vol = (long)L->nx * L->ny * L->nz;
    for (long n = 0; n < vol; ++n) {
        double fn[ORC3_MAXQ], m[5];
        for (int p = 0; p < q; ++p) fn[p] = f[p * vol + n];
        orc3_node_moments(L, fn, m);
        for (int k = 0; k < 5; ++k) out[k * vol + n] = m[k];
    }
}

/* Global sums (compensated): mass, momentum x, y, z, energy sum |v|^2 f. */
void orc3_conserved(const orc_lattice3 *L, const double *f, double *out)
{
    const int q1 = L->q1;
    const long vol = (long)L->nx * L->ny * L->nz;
    double s[5] = {0, 0, 0, 0, 0}, c[5] = {0, 0, 0, 0, 0};
    for (int a = 0; a < q1; ++a)
        for (int b = 0; b < q1; ++b)
            for (int k = 0; k < q1; ++k) {
                const int p = (a * q1 + b) * q1 + k;
                const double cx = L->v[a], cy = L->v[b], cz = L->v[k];
                for (long n = 0; n < vol; ++n) {
                    const double fv = f[p * vol + n];
                    neu_add(&s[0], &c[0], fv);
                    neu_add(&s[1], &c[1], cx * fv);
                    neu_add(&s[2], &c[2], cy * fv);
                    neu_add(&s[3], &c[3], cz * fv);
                    neu_add(&s[4], &c[4], (cx * cx + cy * cy + cz * cz) * fv);
                }
            }
    for (int k = 0; k < 5; ++k) out[k] = s[k] + c[k];
}

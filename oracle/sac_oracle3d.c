/*
 * sac_oracle3d.c -- plain, slow FP64 CPU oracle of the 3D form of the same
 * ideal-MHD step (SMAUG+, arXiv 1710.06423: section 2 writes the equations for
 * vector fields; the paper runs them in 2D and names 3D as the natural
 * extension).  TEST INFRASTRUCTURE ONLY: nothing on the product path may link,
 * load or call this file.  It shares no code with the CUDA library.
 *
 * Eight conserved fields rho, m_x, m_y, m_z, e, B_x, B_y, B_z (no background,
 * no gravity), periodic boundaries, ghost width 3.  Every operator is the 2D
 * oracle's, applied along x, y and z, and every sum over directions adds the z
 * term last in the 2D order:
 *   p_k = (g-1)(e - m.v/2 - |B|^2/2), p_t = p_k + |B|^2/2, m.v and |B|^2 summed
 *     as (x + y) + z;
 *   fluxes along d: F_rho = m_d; F_mk = v_d m_k - B_d B_k + delta_dk p_t;
 *     F_e = v_d (e + p_t) - B_d (B.v); F_Bk = v_d B_k - B_d v_k;
 *   D f_i = (8 (f_{i+1} - f_{i-1}) - (f_{i+2} - f_{i-2})) / (12 d);
 *   hyper-diffusion on faces as in 2D (d1, d3, R = max3|d3| / max3|d1|,
 *     nu = c2 d cmax_d R + c_shk d d s_f, s = max(0, -((D_x v_x + D_y v_y) + D_z v_z)));
 *   k = ((H_x + H_y) + H_z) - ((D_x F_x + D_y F_y) + D_z F_z);
 *   c_fast^2 = (gamma p_k + |B|^2)/rho, cmax_d = max(|v_d| + c_fast);
 *   dt = C min(min(dx/cmax_x, dy/cmax_y), dz/cmax_z);
 *   classical RK4.
 * A z-uniform state with m_z = B_z = 0 therefore gives the 2D oracle's values
 * bit for bit (each z term is an exact zero).
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared [-fopenmp].
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define NF3 8
#define GH 3

typedef struct {
    int nx, ny, nz;
    double dx, dy, dz;
    double gamma;
    double courant;
    int hyperdiffusion;
    double c2[NF3];
    double c_shk;
    int nthreads;
} orc3_params;

static int wrap3(int i, int n) { int r = i % n; return r < 0 ? r + n : r; }

static void set_threads3(const orc3_params *p)
{
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    omp_set_num_threads(p->nthreads > 0 ? p->nthreads : 1);
#else
    (void)p;
#endif
}

#define EX3(p) ((size_t)(p)->nx + 2 * GH)
#define EY3(p) ((size_t)(p)->ny + 2 * GH)
#define EZ3(p) ((size_t)(p)->nz + 2 * GH)
#define XI3(p, i, j, k) ((((size_t)((k) + GH)) * EY3(p) + (size_t)((j) + GH)) * EX3(p) + (size_t)((i) + GH))

size_t orc3_ext_size(const orc3_params *p) { return EX3(p) * EY3(p) * EZ3(p); }

/* ghost-extended copy of one periodic field [nz][ny][nx] */
static void extend_periodic(const orc3_params *p, const double *a, double *e)
{
    for (int k = -GH; k < p->nz + GH; ++k)
        for (int j = -GH; j < p->ny + GH; ++j)
            for (int i = -GH; i < p->nx + GH; ++i)
                e[XI3(p, i, j, k)] = a[((size_t)wrap3(k, p->nz) * p->ny + wrap3(j, p->ny)) * p->nx + wrap3(i, p->nx)];
}

static double dcen3(const double *f, size_t c, size_t s, double d12)
{
    return (8.0 * (f[c + s] - f[c - s]) - (f[c + 2 * s] - f[c - 2 * s])) / d12;
}

void orc3_rhs(const orc3_params *p, const double *w, double cmax_x, double cmax_y, double cmax_z, double *kout)
{
    const size_t n = (size_t)p->nx * p->ny * p->nz, ne = orc3_ext_size(p);
    const size_t st[3] = {1, EX3(p), EX3(p) * EY3(p)};
    const double gm1 = p->gamma - 1.0;
    set_threads3(p);
    double *u = calloc(NF3 * ne, sizeof(double));
    double *v = calloc(3 * ne, sizeof(double));
    double *fl = calloc(3 * NF3 * ne, sizeof(double));   /* fluxes [d][f] */
    double *s = calloc(ne, sizeof(double));
    for (int f = 0; f < NF3; ++f) extend_periodic(p, w + f * n, u + f * ne);
    const double *rt = u, *mx = u + ne, *my = u + 2 * ne, *mz = u + 3 * ne, *et = u + 4 * ne,
                 *bx = u + 5 * ne, *by = u + 6 * ne, *bz = u + 7 * ne;

    #pragma omp parallel for schedule(static)
    for (long c = 0; c < (long)ne; ++c) {
        double rho = rt[c];
        double ux = mx[c] / rho, uy = my[c] / rho, uz = mz[c] / rho;
        double ekin = 0.5 * ((mx[c] * ux + my[c] * uy) + mz[c] * uz);
        double b2 = 0.5 * ((bx[c] * bx[c] + by[c] * by[c]) + bz[c] * bz[c]);
        double pk = gm1 * ((et[c] - ekin) - b2);
        double pt = pk + b2;
        double bv = (bx[c] * ux + by[c] * uy) + bz[c] * uz;
        double etot = et[c] + pt;
        v[c] = ux; v[ne + c] = uy; v[2 * ne + c] = uz;
        const double ud[3] = {ux, uy, uz};
        const double bd[3] = {bx[c], by[c], bz[c]};
        const double md[3] = {mx[c], my[c], mz[c]};
        for (int d = 0; d < 3; ++d) {
            double *F = fl + (size_t)d * NF3 * ne;
            F[0 * ne + c] = md[d];
            for (int q = 0; q < 3; ++q) {
                double f = ud[d] * md[q] - bd[d] * bd[q];
                F[(1 + q) * ne + c] = (q == d) ? f + pt : f;
            }
            F[4 * ne + c] = ud[d] * etot - bd[d] * bv;
            for (int q = 0; q < 3; ++q) F[(5 + q) * ne + c] = ud[d] * bd[q] - bd[d] * ud[q];
        }
    }

    const double dd[3] = {p->dx, p->dy, p->dz};
    const double cm[3] = {cmax_x, cmax_y, cmax_z};
    const int hd = p->hyperdiffusion;
    if (hd) {
        #pragma omp parallel for schedule(static)
        for (int k = -1; k < p->nz + 1; ++k)
            for (int j = -1; j < p->ny + 1; ++j)
                for (int i = -1; i < p->nx + 1; ++i) {
                    size_t c = XI3(p, i, j, k);
                    double div = (dcen3(v, c, st[0], 12.0 * dd[0]) + dcen3(v + ne, c, st[1], 12.0 * dd[1]))
                                 + dcen3(v + 2 * ne, c, st[2], 12.0 * dd[2]);
                    s[c] = fmax(0.0, -div);
                }
    }

    #pragma omp parallel for schedule(static)
    for (int k = 0; k < p->nz; ++k)
        for (int j = 0; j < p->ny; ++j)
            for (int i = 0; i < p->nx; ++i) {
                size_t c = XI3(p, i, j, k);
                for (int f = 0; f < NF3; ++f) {
                    const double *uf = u + f * ne;
                    double hsum = 0.0;
                    if (hd) {
                        for (int d = 0; d < 3; ++d) {
                            size_t S = st[d];
                            double a = (p->c2[f] * dd[d]) * cm[d];
                            double bsh = (p->c_shk * dd[d]) * dd[d];
                            double g[2];
                            for (int side = 0; side < 2; ++side) {
                                size_t fc = side ? c : c - S;
                                double a1[3], a3[3], d1c = 0.0;
                                for (int o = -1; o <= 1; ++o) {
                                    size_t q = (o < 0) ? fc - S : (o > 0 ? fc + S : fc);
                                    double d1 = uf[q + S] - uf[q];
                                    double d3 = (uf[q + 2 * S] - uf[q - S]) - 3.0 * d1;
                                    a1[o + 1] = fabs(d1);
                                    a3[o + 1] = fabs(d3);
                                    if (o == 0) d1c = d1;
                                }
                                double m1 = fmax(fmax(a1[0], a1[1]), a1[2]);
                                double m3 = fmax(fmax(a3[0], a3[1]), a3[2]);
                                double r = (m1 > 0.0) ? m3 / m1 : 0.0;
                                double sf = 0.5 * (s[fc] + s[fc + S]);
                                double nu = a * r + bsh * sf;
                                g[side] = nu * d1c;
                            }
                            hsum = hsum + (g[1] - g[0]) / (dd[d] * dd[d]);
                        }
                    }
                    double dfx = dcen3(fl + (0 * NF3 + f) * ne, c, st[0], 12.0 * dd[0]);
                    double dfy = dcen3(fl + (1 * NF3 + f) * ne, c, st[1], 12.0 * dd[1]);
                    double dfz = dcen3(fl + (2 * NF3 + f) * ne, c, st[2], 12.0 * dd[2]);
                    kout[f * n + ((size_t)k * p->ny + j) * p->nx + i] = hsum - ((dfx + dfy) + dfz);
                }
            }
    free(u); free(v); free(fl); free(s);
}

void orc3_cmax(const orc3_params *p, const double *w, double *cx, double *cy, double *cz)
{
    const size_t n = (size_t)p->nx * p->ny * p->nz;
    const double gm1 = p->gamma - 1.0;
    double ax = 0.0, ay = 0.0, az = 0.0;
    for (size_t c = 0; c < n; ++c) {
        double rho = w[c], mx = w[n + c], my = w[2 * n + c], mz = w[3 * n + c], et = w[4 * n + c];
        double bx = w[5 * n + c], by = w[6 * n + c], bz = w[7 * n + c];
        double ux = mx / rho, uy = my / rho, uz = mz / rho;
        double ekin = 0.5 * ((mx * ux + my * uy) + mz * uz);
        double b2 = 0.5 * ((bx * bx + by * by) + bz * bz);
        double pk = gm1 * ((et - ekin) - b2);
        double cf = sqrt((p->gamma * pk + ((bx * bx + by * by) + bz * bz)) / rho);
        double sx = fabs(ux) + cf, sy = fabs(uy) + cf, sz = fabs(uz) + cf;
        if (!(sx <= ax)) ax = sx;   /* NaN propagates */
        if (!(sy <= ay)) ay = sy;
        if (!(sz <= az)) az = sz;
    }
    *cx = ax; *cy = ay; *cz = az;
}


/*
 * Discrete divergence of B per cell (section 2's fourth-order central
 * difference, the one the flux derivatives use, in each of the three
 * directions; periodic box):
 *     div = Dx(Bx) + Dy(By) + Dz(Bz),
 *     Dx(f)(i) = (f(i-2) - 8 f(i-1) + 8 f(i+1) - f(i+2)) / (12 dx),
 * neighbours wrapped across the box.  div has the layout of one field,
 * [nz][ny][nx].
 */
void orc3_divb(const orc3_params *p, const double *w, double *div)
{
    const int nx = p->nx, ny = p->ny, nz = p->nz;
    const size_t n = (size_t)nx * ny * nz;
    const double *bx = w + 5 * n, *by = w + 6 * n, *bz = w + 7 * n;
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double fx[5], fy[5], fz[5];
                for (int o = -2; o <= 2; ++o) {
                    fx[o + 2] = bx[((size_t)k * ny + j) * nx + wrap3(i + o, nx)];
                    fy[o + 2] = by[((size_t)k * ny + wrap3(j + o, ny)) * nx + i];
                    fz[o + 2] = bz[((size_t)wrap3(k + o, nz) * ny + j) * nx + i];
                }
                const double dxb = (fx[0] - 8.0 * fx[1] + 8.0 * fx[3] - fx[4]) / (12.0 * p->dx);
                const double dyb = (fy[0] - 8.0 * fy[1] + 8.0 * fy[3] - fy[4]) / (12.0 * p->dy);
                const double dzb = (fz[0] - 8.0 * fz[1] + 8.0 * fz[3] - fz[4]) / (12.0 * p->dz);
                div[((size_t)k * ny + j) * nx + i] = (dxb + dyb) + dzb;
            }
}

double orc3_cfl_dt(const orc3_params *p, double cx, double cy, double cz)
{
    return p->courant * fmin(fmin(p->dx / cx, p->dy / cy), p->dz / cz);
}

void orc3_rk4_step(const orc3_params *p, double *w, double dt, double cx, double cy, double cz)
{
    const size_t m = (size_t)NF3 * p->nx * p->ny * p->nz;
    double *k1 = malloc(m * sizeof(double)), *k2 = malloc(m * sizeof(double));
    double *k3 = malloc(m * sizeof(double)), *k4 = malloc(m * sizeof(double));
    double *us = malloc(m * sizeof(double));
    const double h = 0.5 * dt, d6 = dt / 6.0;
    orc3_rhs(p, w, cx, cy, cz, k1);
    for (size_t c = 0; c < m; ++c) us[c] = w[c] + h * k1[c];
    orc3_rhs(p, us, cx, cy, cz, k2);
    for (size_t c = 0; c < m; ++c) us[c] = w[c] + h * k2[c];
    orc3_rhs(p, us, cx, cy, cz, k3);
    for (size_t c = 0; c < m; ++c) us[c] = w[c] + dt * k3[c];
    orc3_rhs(p, us, cx, cy, cz, k4);
    for (size_t c = 0; c < m; ++c) w[c] = w[c] + d6 * (((k1[c] + 2.0 * k2[c]) + 2.0 * k3[c]) + k4[c]);
    free(k1); free(k2); free(k3); free(k4); free(us);
}

/* CFL steps (or fixed_dt > 0) until max_steps; returns 0, or -1 on a non-finite step */
int orc3_run(const orc3_params *p, double *w, double *t, long max_steps, double fixed_dt, long *steps)
{
    long n = 0;
    for (; n < max_steps; ++n) {
        double cx, cy, cz;
        orc3_cmax(p, w, &cx, &cy, &cz);
        double dt = fixed_dt > 0.0 ? fixed_dt : orc3_cfl_dt(p, cx, cy, cz);
        if (!(dt > 0.0) || !isfinite(dt)) { *steps = n; return -1; }
        orc3_rk4_step(p, w, dt, cx, cy, cz);
        *t += dt;
    }
    *steps = n;
    return 0;
}

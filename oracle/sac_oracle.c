/*
 * sac_oracle.c -- plain, slow FP64 CPU oracle of the SAC-family 2D ideal-MHD
 * step (SMAUG+, arXiv 1710.06423).  TEST INFRASTRUCTURE ONLY: nothing on the
 * product path may link, load or call this file.  It shares no code, header,
 * table or constant generator with the CUDA library.
 *
 * What it computes, in the paper's order (section 2, "Numerical Approach"):
 *   - the conservative ideal-MHD system (section 2 equations: mass, momentum,
 *     energy, induction) with total pressure p_t = p_k + B^2/2 and kinetic
 *     pressure p_k = (gamma-1)(e - rho v^2/2 - B^2/2), units with mu0 = 1;
 *   - written in perturbation/background split form (section 2 "with
 *     stratification"; the split itself is deferred by the paper to SAC/SMAUG,
 *     the reading used here is stated below);
 *   - fourth-order central differences of the fluxes (section 2);
 *   - hyper-diffusion / hyper-resistivity whose coefficient is the ratio of the
 *     third-order to the first-order difference of each variable, scaled by the
 *     maximum wave speed, plus a shock viscosity that grows with compression
 *     (section 2, the two paragraphs after the equations);
 *   - classical fourth-order Runge-Kutta in time (section 2);
 *   - the maximum signal speed over the domain, which sets both the
 *     hyper-viscosity scale and the CFL time step (section 2).
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   * split form: rho = rho_b + rt, B = B_b + Bt, m = rho v (background at rest);
 *     pt_k = (g-1)(et - m.v/2 - B_b.Bt - |Bt|^2/2), pt_t = pt_k + B_b.Bt + |Bt|^2/2;
 *     p_kb = (g-1)(e_b - |B_b|^2/2), p_tb = p_kb + |B_b|^2/2.
 *   * fluxes along d: F_rho = m_d;
 *       F_mk = v_d m_k - (Bt_d Bt_k + Bt_d Bb_k + Bb_d Bt_k) + delta_dk pt_t;
 *       F_e  = v_d (et + e_b + pt_t + p_tb) - B_d (B.v);
 *       F_Bk = v_d B_k - B_d v_k  (full B).
 *     The energy equation of section 2 carries a stray "+grad p_t" term and
 *     writes rho g for rho g; both are read as typos.
 *   * D f_i = (8 (f_{i+1} - f_{i-1}) - (f_{i+2} - f_{i-2})) / (12 dx).
 *   * hyper-diffusion of every conserved u along d, on faces f = i+1/2:
 *       d1_f = u_{i+1} - u_i,  d3_f = (u_{i+2} - u_{i-1}) - 3 d1_f,
 *       R_f = max3|d3| / max3|d1| over faces f-1, f, f+1 (0 if the max |d1| is 0),
 *       s_i = max(0, -(D_x v_x + D_y v_y)_i),  s_f = (s_i + s_{i+1}) / 2,
 *       nu_f = (c2_u dx cmax_d) R_f + (c_shk dx dx) s_f,
 *       H_i = (nu_{i+1/2} d1_{i+1/2} - nu_{i-1/2} d1_{i-1/2}) / (dx dx).
 *     single-face variant (hd_single_face = 1, the minimal form of the same
 *     section-2 description, stencil radius 2): R_f = |d3_f| / |d1_f| on the
 *     face itself (0 if d1_f = 0).
 *   * k_u = (H_x + H_y) - (D_x F_x + D_y F_y).
 *   * gravity g (section 2: the rho g source of the momentum equation and its
 *     work term in the energy equation), with the background read as being in
 *     magnetohydrostatic balance, -grad p_tb + div(B_b B_b) + rho_b g = 0, so
 *     that its own force cancels: the perturbation sources are
 *       S_mk = rt g_k,  S_e = m.g = m_x g_x + m_y g_y  (m the total momentum),
 *     added last: k = ((H_x + H_y) - (D_x F_x + D_y F_y)) + S, and only when
 *     g is nonzero.
 *   * c_fast^2 = (gamma p_k + |B|^2)/rho with total p_k; cmax_d = max(|v_d| + c_fast)
 *     over interior cells, taken once per step from the step-start state and
 *     used by all four stages; dt = C min(dx/cmax_x, dy/cmax_y).
 *   * boundaries (ghost width 3): periodic = wrapped interior; outflow = nearest
 *     interior cell of the current stage state; fixed = nearest interior cell of
 *     the state the run started from, held.  Ghosts are filled along x for the
 *     interior rows first, then along y for every column (corners included).
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared [-fopenmp].  No FMA
 * contraction, IEEE division and square root, round to nearest.  OpenMP only
 * splits the outer row loops; each value is computed by the same expression in
 * the same order whatever the thread count.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define NF 6   /* conserved perturbation fields: rt, mx, my, et, btx, bty */
#define NB 4   /* background fields: rho_b, e_b, bbx, bby */
#define GH 3   /* ghost width */

enum { BC_PERIODIC = 0, BC_FIXED = 1, BC_OUTFLOW = 2 };

typedef struct {
    int nx, ny;
    double dx, dy;
    double gamma;
    double courant;
    int bc_x, bc_y;
    int hyperdiffusion;   /* 0: ideal fluxes only (no hyper-diffusion, no shock viscosity) */
    double c2[NF];        /* hyper-diffusion coefficient per conserved variable */
    double c_shk;         /* shock-viscosity coefficient */
    int nthreads;         /* OpenMP threads (<= 0: 1) */
    double grav[2];       /* gravitational acceleration (g_x, g_y); zero: no source */
    int hd_single_face;   /* 1: hyper-diffusion ratio from the face itself, not the max over 3 faces */
} orc_params;

/* ghost-extended index: i in [-GH, nx+GH), j in [-GH, ny+GH) */
#define EX(p) ((p)->nx + 2 * GH)
#define EY(p) ((p)->ny + 2 * GH)
#define XI(p, i, j) ((size_t)((j) + GH) * (size_t)EX(p) + (size_t)((i) + GH))

static int wrap(int i, int n) { int r = i % n; return r < 0 ? r + n : r; }
static int clampi(int i, int n) { return i < 0 ? 0 : (i >= n ? n - 1 : i); }

static void set_threads(const orc_params *p)
{
#ifdef _OPENMP
    extern void omp_set_num_threads(int);
    omp_set_num_threads(p->nthreads > 0 ? p->nthreads : 1);
#else
    (void)p;
#endif
}

/*
 * Fill one ghost-extended field `e` whose interior is already set.
 * `held` (same shape, may be NULL when no direction is fixed) supplies ghost
 * values of fixed directions.  Order: x ghosts of interior rows, then y ghosts
 * of all columns.
 */
static void fill_ghosts(const orc_params *p, double *e, const double *held)
{
    int nx = p->nx, ny = p->ny;
    for (int j = 0; j < ny; ++j) {
        for (int g = 1; g <= GH; ++g) {
            int il = -g, ir = nx - 1 + g;
            if (p->bc_x == BC_PERIODIC) {
                e[XI(p, il, j)] = e[XI(p, wrap(il, nx), j)];
                e[XI(p, ir, j)] = e[XI(p, wrap(ir, nx), j)];
            } else if (p->bc_x == BC_OUTFLOW) {
                e[XI(p, il, j)] = e[XI(p, 0, j)];
                e[XI(p, ir, j)] = e[XI(p, nx - 1, j)];
            } else {
                e[XI(p, il, j)] = held[XI(p, il, j)];
                e[XI(p, ir, j)] = held[XI(p, ir, j)];
            }
        }
    }
    for (int i = -GH; i < nx + GH; ++i) {
        for (int g = 1; g <= GH; ++g) {
            int jb = -g, jt = ny - 1 + g;
            if (p->bc_y == BC_PERIODIC) {
                e[XI(p, i, jb)] = e[XI(p, i, wrap(jb, ny))];
                e[XI(p, i, jt)] = e[XI(p, i, wrap(jt, ny))];
            } else if (p->bc_y == BC_OUTFLOW) {
                e[XI(p, i, jb)] = e[XI(p, i, 0)];
                e[XI(p, i, jt)] = e[XI(p, i, ny - 1)];
            } else {
                e[XI(p, i, jb)] = held[XI(p, i, jb)];
                e[XI(p, i, jt)] = held[XI(p, i, jt)];
            }
        }
    }
}

/* Copy interior [ny][nx] into a ghost-extended array (ghosts untouched). */
static void put_interior(const orc_params *p, double *e, const double *a)
{
    for (int j = 0; j < p->ny; ++j)
        for (int i = 0; i < p->nx; ++i)
            e[XI(p, i, j)] = a[(size_t)j * p->nx + i];
}

/*
 * Held ghost values of a run, from its starting state w0 [NF][ny][nx]:
 * `held` is NF ghost-extended fields whose ghosts follow the nearest-interior
 * rule in fixed directions and the periodic rule in periodic directions.
 */
void orc_make_held(const orc_params *p, const double *w0, double *held)
{
    size_t n = (size_t)p->nx * p->ny, ne = (size_t)EX(p) * EY(p);
    orc_params q = *p;
    if (q.bc_x == BC_FIXED) q.bc_x = BC_OUTFLOW;
    if (q.bc_y == BC_FIXED) q.bc_y = BC_OUTFLOW;
    for (int f = 0; f < NF; ++f) {
        double *e = held + f * ne;
        memset(e, 0, ne * sizeof(double));
        put_interior(p, e, w0 + f * n);
        fill_ghosts(&q, e, NULL);
    }
}

size_t orc_ext_size(const orc_params *p) { return (size_t)EX(p) * EY(p); }

/* Fourth-order central difference (section 2) at ghost-extended index c, stride s. */
static double dcen(const double *f, size_t c, size_t s, double d12)
{
    return (8.0 * (f[c + s] - f[c - s]) - (f[c + 2 * s] - f[c - 2 * s])) / d12;
}

/*
 * Right-hand side k = f(w) of the split system.
 *   w    [NF][ny][nx] conserved perturbations (interior only)
 *   bg   [NB][ny][nx] background (rho_b, e_b, bbx, bby) or NULL (identically 0)
 *   held ghost-extended held values (orc_make_held) or NULL if no fixed side
 *   cmax_x, cmax_y: maximum signal speeds of the step (hyper-diffusion scale)
 *   k    [NF][ny][nx] output
 */
void orc_rhs(const orc_params *p, const double *w, const double *bg,
             const double *held, double cmax_x, double cmax_y, double *k)
{
    const int nx = p->nx, ny = p->ny;
    const size_t n = (size_t)nx * ny, ne = orc_ext_size(p);
    const size_t sx = 1, sy = (size_t)EX(p);
    const double gm1 = p->gamma - 1.0;

    set_threads(p);
    double *u = calloc(NF * ne, sizeof(double));      /* conserved, with ghosts */
    double *b = calloc(NB * ne, sizeof(double));      /* background, with ghosts */
    double *vx = calloc(ne, sizeof(double)), *vy = calloc(ne, sizeof(double));
    double *ptt = calloc(ne, sizeof(double));         /* perturbed total pressure */
    double *ptb = calloc(ne, sizeof(double));         /* background total pressure */
    double *fx = calloc(NF * ne, sizeof(double)), *fy = calloc(NF * ne, sizeof(double));
    double *s = calloc(ne, sizeof(double));           /* shock indicator */

    for (int f = 0; f < NF; ++f) {
        put_interior(p, u + f * ne, w + f * n);
        fill_ghosts(p, u + f * ne, held ? held + f * ne : NULL);
    }
    if (bg) {
        /* the background is static; its ghosts follow the same rules, with a
           fixed side read as "nearest interior" of the background itself */
        orc_params q = *p;
        if (q.bc_x == BC_FIXED) q.bc_x = BC_OUTFLOW;
        if (q.bc_y == BC_FIXED) q.bc_y = BC_OUTFLOW;
        for (int f = 0; f < NB; ++f) {
            put_interior(p, b + f * ne, bg + f * n);
            fill_ghosts(&q, b + f * ne, NULL);
        }
    }
    const double *rt = u, *mx = u + ne, *my = u + 2 * ne, *et = u + 3 * ne,
                 *btx = u + 4 * ne, *bty = u + 5 * ne;
    const double *rb = b, *eb = b + ne, *bbx = b + 2 * ne, *bby = b + 3 * ne;

    /* primitives and fluxes at every ghost-extended cell (section 2 equations) */
    #pragma omp parallel for schedule(static)
    for (int jj = 0; jj < EY(p); ++jj) {
        for (int ii = 0; ii < EX(p); ++ii) {
            size_t c = (size_t)jj * EX(p) + ii;
            double rho = rb[c] + rt[c];
            double ux = mx[c] / rho, uy = my[c] / rho;
            double ekin = 0.5 * (mx[c] * ux + my[c] * uy);
            double bb = bbx[c] * btx[c] + bby[c] * bty[c];
            double b2p = 0.5 * (btx[c] * btx[c] + bty[c] * bty[c]);
            double pk = gm1 * (((et[c] - ekin) - bb) - b2p);
            double pt = (pk + bb) + b2p;
            double b2b = 0.5 * (bbx[c] * bbx[c] + bby[c] * bby[c]);
            double pkb = gm1 * (eb[c] - b2b);
            double ptbk = pkb + b2b;
            double bx = bbx[c] + btx[c], by = bby[c] + bty[c];
            double bv = bx * ux + by * uy;
            double etot = ((et[c] + eb[c]) + pt) + ptbk;
            vx[c] = ux; vy[c] = uy; ptt[c] = pt; ptb[c] = ptbk;
            /* x fluxes */
            fx[0 * ne + c] = mx[c];
            fx[1 * ne + c] = (ux * mx[c] - ((btx[c] * btx[c] + btx[c] * bbx[c]) + bbx[c] * btx[c])) + pt;
            fx[2 * ne + c] = ux * my[c] - ((btx[c] * bty[c] + btx[c] * bby[c]) + bbx[c] * bty[c]);
            fx[3 * ne + c] = ux * etot - bx * bv;
            fx[4 * ne + c] = ux * bx - bx * ux;
            fx[5 * ne + c] = ux * by - bx * uy;
            /* y fluxes */
            fy[0 * ne + c] = my[c];
            fy[1 * ne + c] = uy * mx[c] - ((bty[c] * btx[c] + bty[c] * bbx[c]) + bby[c] * btx[c]);
            fy[2 * ne + c] = (uy * my[c] - ((bty[c] * bty[c] + bty[c] * bby[c]) + bby[c] * bty[c])) + pt;
            fy[3 * ne + c] = uy * etot - by * bv;
            fy[4 * ne + c] = uy * bx - by * ux;
            fy[5 * ne + c] = uy * by - by * uy;
        }
    }

    const double d12x = 12.0 * p->dx, d12y = 12.0 * p->dy;
    const int hd = p->hyperdiffusion;

    /* shock indicator s = max(0, -div v) where both centred differences fit */
    if (hd) {
        #pragma omp parallel for schedule(static)
        for (int j = -1; j < ny + 1; ++j) {
            for (int i = -1; i < nx + 1; ++i) {
                size_t c = XI(p, i, j);
                double div = dcen(vx, c, sx, d12x) + dcen(vy, c, sy, d12y);
                s[c] = fmax(0.0, -div);
            }
        }
    }

    const double cm[2] = {cmax_x, cmax_y};
    const int grav = p->grav[0] != 0.0 || p->grav[1] != 0.0;
    const double dd[2] = {p->dx, p->dy};
    const size_t st[2] = {sx, sy};

    #pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            size_t c = XI(p, i, j);
            for (int f = 0; f < NF; ++f) {
                const double *uf = u + f * ne;
                double hsum = 0.0;
                if (hd) {
                    for (int d = 0; d < 2; ++d) {
                        size_t S = st[d];
                        double a = (p->c2[f] * dd[d]) * cm[d];
                        double bsh = (p->c_shk * dd[d]) * dd[d];
                        double gface[2];
                        /* faces i-1/2 (base cell c-S) and i+1/2 (base cell c) */
                        for (int side = 0; side < 2; ++side) {
                            size_t fc = side ? c : c - S;   /* face between fc and fc+S */
                            double a1[3], a3[3], d1c = 0.0;
                            for (int o = -1; o <= 1; ++o) {
                                size_t q = (o < 0) ? fc - S : (o > 0 ? fc + S : fc);
                                double d1 = uf[q + S] - uf[q];
                                double d3 = (uf[q + 2 * S] - uf[q - S]) - 3.0 * d1;
                                a1[o + 1] = fabs(d1);
                                a3[o + 1] = fabs(d3);
                                if (o == 0) d1c = d1;
                            }
                            double m1 = p->hd_single_face ? a1[1] : fmax(fmax(a1[0], a1[1]), a1[2]);
                            double m3 = p->hd_single_face ? a3[1] : fmax(fmax(a3[0], a3[1]), a3[2]);
                            double r = (m1 > 0.0) ? m3 / m1 : 0.0;
                            double sf = 0.5 * (s[fc] + s[fc + S]);
                            double nu = a * r + bsh * sf;
                            gface[side] = nu * d1c;
                        }
                        double h = (gface[1] - gface[0]) / (dd[d] * dd[d]);
                        hsum = hsum + h;
                    }
                }
                double dfx = dcen(fx + f * ne, c, sx, d12x);
                double dfy = dcen(fy + f * ne, c, sy, d12y);
                double kf = hsum - (dfx + dfy);
                if (grav) {
                    if (f == 1) kf = kf + rt[c] * p->grav[0];
                    else if (f == 2) kf = kf + rt[c] * p->grav[1];
                    else if (f == 3) kf = kf + (mx[c] * p->grav[0] + my[c] * p->grav[1]);
                }
                k[f * n + (size_t)j * nx + i] = kf;
            }
        }
    }
    (void)ptt; (void)ptb;
    free(u); free(b); free(vx); free(vy); free(ptt); free(ptb);
    free(fx); free(fy); free(s);
}

/*
 * Maximum signal speed per direction over the interior (section 2: the
 * hyper-viscosity and the time step need the largest wave speed in the domain):
 * cmax_d = max(|v_d| + sqrt((gamma p_k + |B|^2) / rho)), total p_k and B.
 * A NaN anywhere makes the result NaN.
 */
void orc_cmax(const orc_params *p, const double *w, const double *bg,
              double *cmax_x, double *cmax_y)
{
    const size_t n = (size_t)p->nx * p->ny;
    const double gm1 = p->gamma - 1.0;
    double cx = 0.0, cy = 0.0;
    for (size_t c = 0; c < n; ++c) {
        double r = w[c], mx = w[n + c], my = w[2 * n + c], et = w[3 * n + c];
        double btx = w[4 * n + c], bty = w[5 * n + c];
        double rb = 0, eb = 0, bbx = 0, bby = 0;
        if (bg) { rb = bg[c]; eb = bg[n + c]; bbx = bg[2 * n + c]; bby = bg[3 * n + c]; }
        double rho = rb + r;
        double ux = mx / rho, uy = my / rho;
        double ekin = 0.5 * (mx * ux + my * uy);
        double bb = bbx * btx + bby * bty;
        double b2p = 0.5 * (btx * btx + bty * bty);
        double pk = gm1 * (((et - ekin) - bb) - b2p);
        double b2b = 0.5 * (bbx * bbx + bby * bby);
        double pkb = gm1 * (eb - b2b);
        double pkt = pkb + pk;
        double bx = bbx + btx, by = bby + bty;
        double cf = sqrt((p->gamma * pkt + (bx * bx + by * by)) / rho);
        double sx = fabs(ux) + cf, sy = fabs(uy) + cf;
        if (!(sx <= cx)) cx = sx;   /* NaN propagates */
        if (!(sy <= cy)) cy = sy;
    }
    *cmax_x = cx;
    *cmax_y = cy;
}

/*
 * Discrete divergence of the total field B = B_b + Bt (section 2: the split
 * form carries B in two parts and the scheme differences each flux with the
 * fourth-order central formula), per interior cell:
 *     div[j][i] = Dx(Bx)(i, j) + Dy(By)(i, j),
 *     Dx(f)(i) = (f(i-2) - 8 f(i-1) + 8 f(i+1) - f(i+2)) / (12 dx),
 * the neighbours taken inside the interior, wrapped across periodic sides.
 * mask[j][i] = 1 where every neighbour exists that way (a non-periodic side
 * leaves out the two cells next to it), else 0 and div = 0 there.  A
 * direction of one cell has no derivative (that term is 0).
 */
void orc_divb(const orc_params *p, const double *w, const double *bg,
              double *div, unsigned char *mask)
{
    const int nx = p->nx, ny = p->ny;
    const size_t n = (size_t)nx * ny;
    for (int j = 0; j < ny; ++j) {
        for (int i = 0; i < nx; ++i) {
            const size_t c = (size_t)j * nx + i;
            int ok = 1;
            if (nx > 1 && p->bc_x != BC_PERIODIC && (i < 2 || i > nx - 3)) ok = 0;
            if (ny > 1 && p->bc_y != BC_PERIODIC && (j < 2 || j > ny - 3)) ok = 0;
            mask[c] = (unsigned char)ok;
            div[c] = 0.0;
            if (!ok) continue;
            double d = 0.0;
            if (nx > 1) {
                double f[5];
                for (int k = -2; k <= 2; ++k) {
                    size_t s = (size_t)j * nx + wrap(i + k, nx);
                    f[k + 2] = w[4 * n + s] + (bg ? bg[2 * n + s] : 0.0);
                }
                d += (f[0] - 8.0 * f[1] + 8.0 * f[3] - f[4]) / (12.0 * p->dx);
            }
            if (ny > 1) {
                double f[5];
                for (int k = -2; k <= 2; ++k) {
                    size_t s = (size_t)wrap(j + k, ny) * nx + i;
                    f[k + 2] = w[5 * n + s] + (bg ? bg[3 * n + s] : 0.0);
                }
                d += (f[0] - 8.0 * f[1] + 8.0 * f[3] - f[4]) / (12.0 * p->dy);
            }
            div[c] = d;
        }
    }
}

/* CFL time step from the signal speeds: dt = C min(dx/cmax_x, dy/cmax_y). */
double orc_cfl_dt(const orc_params *p, double cmax_x, double cmax_y)
{
    double tx = p->dx / cmax_x, ty = p->dy / cmax_y;
    return p->courant * fmin(tx, ty);
}

/*
 * One classical RK4 step (section 2) of size dt with the step's signal speeds:
 *   k1 = f(U0), U1 = U0 + (dt/2) k1, k2 = f(U1), U2 = U0 + (dt/2) k2,
 *   k3 = f(U2), U3 = U0 + dt k3,     k4 = f(U3),
 *   U  = U0 + (dt/6) (((k1 + 2 k2) + 2 k3) + k4).
 * w is updated in place.
 */
void orc_rk4_step(const orc_params *p, double *w, const double *bg,
                  const double *held, double dt, double cmax_x, double cmax_y)
{
    const size_t n = (size_t)p->nx * p->ny, m = NF * n;
    double *k1 = malloc(m * sizeof(double)), *k2 = malloc(m * sizeof(double));
    double *k3 = malloc(m * sizeof(double)), *k4 = malloc(m * sizeof(double));
    double *us = malloc(m * sizeof(double));
    const double h = 0.5 * dt, d6 = dt / 6.0;

    orc_rhs(p, w, bg, held, cmax_x, cmax_y, k1);
    for (size_t c = 0; c < m; ++c) us[c] = w[c] + h * k1[c];
    orc_rhs(p, us, bg, held, cmax_x, cmax_y, k2);
    for (size_t c = 0; c < m; ++c) us[c] = w[c] + h * k2[c];
    orc_rhs(p, us, bg, held, cmax_x, cmax_y, k3);
    for (size_t c = 0; c < m; ++c) us[c] = w[c] + dt * k3[c];
    orc_rhs(p, us, bg, held, cmax_x, cmax_y, k4);
    for (size_t c = 0; c < m; ++c)
        w[c] = w[c] + d6 * (((k1[c] + 2.0 * k2[c]) + 2.0 * k3[c]) + k4[c]);
    free(k1); free(k2); free(k3); free(k4); free(us);
}

/*
 * Advance w from time *t toward t_end with CFL steps, at most max_steps steps
 * (max_steps < 0: no limit).  The last step is clipped so that t lands exactly
 * on t_end.  `fixed_dt` > 0 replaces the CFL step (the signal speeds are still
 * taken for the hyper-diffusion).  Returns 0, or -5 when the step size is not
 * finite and positive (NaN state).
 */
int orc_run(const orc_params *p, double *w, const double *bg, const double *held,
            double *t, double t_end, long max_steps, double fixed_dt, long *steps)
{
    long ns = 0;
    double tt = *t;
    while (tt < t_end && (max_steps < 0 || ns < max_steps)) {
        double cx, cy;
        orc_cmax(p, w, bg, &cx, &cy);
        double dt = fixed_dt > 0.0 ? fixed_dt : orc_cfl_dt(p, cx, cy);
        if (!(dt > 0.0) || !isfinite(dt) || !isfinite(cx) || !isfinite(cy)) {
            *t = tt; if (steps) *steps = ns; return -5;
        }
        int last = 0;
        if (tt + dt >= t_end) { dt = t_end - tt; last = 1; }
        orc_rk4_step(p, w, bg, held, dt, cx, cy);
        tt = last ? t_end : tt + dt;
        ++ns;
    }
    *t = tt;
    if (steps) *steps = ns;
    return 0;
}

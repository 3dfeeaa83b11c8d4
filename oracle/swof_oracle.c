/*
 * swof_oracle.c -- plain, slow FP64 CPU oracle of FullSWOF_2D's time step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py may load it.  It shares no code, header,
 * constant or table with the CUDA path; it exists to check that path.
 *
 * What it computes (arXiv 1307.4839, "FullSWOF_Paral"):
 *   - Sec. 2.1, Eq. (SW2D): the 2-D Saint-Venant system, unknowns h, qx = hu,
 *     qy = hv, topography z, rain R, infiltration I, friction S_f.
 *   - Sec. 3.1, Eq. (SW1Dscheme): U* = U - dt/dx [F_{i+1/2L} - F_{i-1/2R} - Fc_i]
 *     applied in x and in y (method of lines, Sec. 2.1 end / Sec. 3 intro).
 *   - Sec. 3.1: hydrostatic reconstruction of the face depths, the
 *     well-balancing corrections S_{i+1/2L}, S_{i-1/2R} and the centred Fc_i.
 *   - Sec. 3.3: the HLL flux with c1 = min, c2 = max of u -+ sqrt(g h) over
 *     U_L and U_R; the CFL condition Eq. (cfl) evaluated on the MUSCL face
 *     values (second order, n_CFL = 0.5).
 *   - Sec. 3.4: MUSCL with the minmod limiter on h, h+z and u (z deduced),
 *     and the discharge-conserving modified velocities.
 *   - Sec. 3.2: semi-implicit friction (given for Darcy-Weisbach; the Manning
 *     law of Sec. 2.1 replaces h by h^{4/3}) and the Heun (SSP-RK2) stages.
 *   - Sec. 3.5: modified Green-Ampt infiltration.
 *   - Algorithm 1: per stage BC -> reconstruction -> hydrostatic ->
 *     flux -> scheme -> friction; then the Heun combine.
 *   - Sec. 2.1: the two friction families, Manning-Strickler (C_f = n^2 or
 *     1/K^2, S_f = C_f |u| u / h^{4/3}) and Darcy-Weisbach-Chezy (C_f =
 *     f/(8g) or 1/C^2, S_f = C_f |u| u / h), each semi-implicit (Sec. 3.2).
 *   - Sec. 2.2: boundary values through ghost cells, the missing ones from
 *     the Riemann invariant that leaves the domain (one imposed variable, h
 *     or q, for a fluvial boundary; both for a torrential inflow).
 *   - Sec. 3.3: the first-order variant (no reconstruction, n_CFL = 1 is
 *     the caller's choice) advanced by one explicit Euler stage.
 *   - Sec. 5.2 (SkelGIS example): the D8 flow direction of a DEM.
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   2-D: F = (hu, hu^2 + g h^2/2, huv), G = (hv, huv, hv^2 + g h^2/2); the
 *   transverse velocity is reconstructed like the normal one; one c1, c2 for
 *   all components.  Dry cells (h <= h_dry) have u = v = 0 and unmodified
 *   face velocities.  dt = n_CFL / (lx/dx + ly/dy) (or n_CFL min(dx/lx,
 *   dy/ly)); dt_max when lx = ly = 0; clamped to rain on/off and t_end.  One
 *   dt per step, reused by both stages.  Manning semi-implicit friction uses
 *   |u| of the stage input and h^{4/3} of the convective output, with
 *   h^{-1/3} from a Newton inverse cube root.  Rain, then Green-Ampt
 *   (A = 1, suction psi > 0: I_C = K_s (1 + (psi + h) dtheta / V_inf),
 *   everything infiltrates while V_inf = 0), then q = 0 where h <= h_dry,
 *   once per step after the Heun combine.  Walls mirror 2 ghost layers
 *   (normal discharge negated), outflow extends the edge cell.  Imposed
 *   boundaries fill both ghost layers with one boundary state built from the
 *   edge cell; the tangential velocity is the edge cell's (imposed h or q) or
 *   zero (both imposed); no switching by flow regime.  First order: face
 *   values are the cell values, one Euler stage per step, the rain /
 *   infiltration / clean-up sequence unchanged.  Gauges record t, h, qx, qy
 *   after every step; the maximum depth is a running max over the states
 *   after each step (starting from the state when tracking is switched on).
 *
 * Rounding order: the expressions below are the ones the CUDA FP64 path must
 * reproduce bit for bit; each is written out plainly (compile with
 * -ffp-contract=off, IEEE division and square root).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    double g, cfl, h_dry, dt_max, t_end;
    int cfl_mode;          /* 0: n_CFL/(lx/dx+ly/dy), 1: n_CFL*min(dx/lx, dy/ly) */
    int bc[4];             /* W, E, S, N: 0 wall, 1 outflow, 2 imposed h,
                              3 imposed discharge, 4 imposed h and discharge */
    int friction;          /* 0 none, 1 Manning, 2 Strickler, 3 Darcy-Weisbach, 4 Chezy */
    double fric_coef;      /* n, K, f or C of that law */
    double rain_rate, rain_t_on, rain_t_off;
    int infiltration;
    double ks, psi, dtheta;
    int check_cfl;         /* count dt > CFL bound of U* */
    double dt_fixed;       /* > 0: fixed dt; a CFL violation is an error */
    int order;             /* 1: first order (Euler); else second order (Heun) */
    double bc_h[4];        /* imposed depth per edge [m] */
    double bc_q[4];        /* imposed discharge per unit width, into the domain [m^2/s] */
} oracle_params;

typedef struct {
    int nx, ny, px, py;
    double dx, dy;
    oracle_params p;
    double *z, *h, *qx, *qy, *h1, *qx1, *qy1, *h2, *qx2, *qy2;
    double *cf;      /* per-cell friction factor C_f (interior), or NULL */
    double p_cf;     /* C_f from the scalar coefficient */
    double *ksmap;   /* per-cell K_s (interior), or NULL */
    double *vinf;    /* infiltrated depth (interior) */
    double *u, *v;   /* cell velocities (padded) */
    /* reconstruction: m = minus side (W or S face of the cell), p = plus side */
    double *xhm, *xhp, *xzm, *xzp, *xum, *xup, *xvm, *xvp;
    double *yhm, *yhp, *yzm, *yzp, *yum, *yup, *yvm, *yvp;
    /* face fluxes; x-face i+1/2 stored at cell i, y-face j+1/2 at cell j */
    double *fx1, *fx2l, *fx2r, *fx3, *fy1, *fy2l, *fy2r, *fy3;
    double t, last_dt, rain_in, infiltrated, outflow;
    long steps, cfl_viol;
    double *dt_seq; int dt_seq_n, dt_seq_pos;
    double *hmax;    /* running max depth (interior), or NULL */
    int *gauge_ij; int n_gauges, gauge_cap, gauge_n;
    double *gauge_rec;   /* [gauge_cap][1 + 3 n_gauges]: t, (h, qx, qy) per gauge */
} oracle_t;

#define IDX(o, i, j) ((size_t)((j) + 2) * (size_t)(o)->px + (size_t)((i) + 2))

/* ---------------- scalar building blocks (Sec. 3.3, 3.4) ---------------- */

/* minmod limiter, Sec. 3.4 */
double oracle_minmod(double a, double b)
{
    if (a >= 0.0 && b >= 0.0) return fmin(a, b);
    if (a <= 0.0 && b <= 0.0) return fmax(a, b);
    return 0.0;
}

/* HLL flux, Sec. 3.3, for one face.  un = normal velocity, ut = transverse
 * velocity (both from the MUSCL-reconstructed face values), hL/hR the
 * hydrostatically reconstructed depths.  F = (normal mass flux, normal
 * momentum flux, transverse momentum flux); the pressure term is included
 * in F[1], the well-balancing corrections are added by the caller. */
void oracle_hll(double g, double hL, double unL, double utL,
                double hR, double unR, double utR, double F[3])
{
    double cL = sqrt(g * hL), cR = sqrt(g * hR);
    double c1 = fmin(unL - cL, unR - cR);
    double c2 = fmax(unL + cL, unR + cR);
    double qL = hL * unL, qR = hR * unR;
    double FL[3], FR[3];
    FL[0] = qL;
    FL[1] = qL * unL + 0.5 * g * hL * hL;
    FL[2] = qL * utL;
    FR[0] = qR;
    FR[1] = qR * unR + 0.5 * g * hR * hR;
    FR[2] = qR * utR;
    if (c1 >= 0.0) {
        F[0] = FL[0]; F[1] = FL[1]; F[2] = FL[2];
    } else if (c2 <= 0.0) {
        F[0] = FR[0]; F[1] = FR[1]; F[2] = FR[2];
    } else {
        double UL[3] = {hL, qL, hL * utL};
        double UR[3] = {hR, qR, hR * utR};
        double r = 1.0 / (c2 - c1);
        double w = c1 * c2 * r;
        for (int k = 0; k < 3; ++k)
            F[k] = (c2 * FL[k] - c1 * FR[k]) * r + w * (UR[k] - UL[k]);
    }
}

/* Inverse cube root x^{-1/3} for x > 0 (normal), by Newton's method on
 * f(y) = y^{-3} - x:  y <- y + y (1 - x y^3) / 3.  The start value comes
 * from the exponent bits: x = m 2^e, m in [1, 2), e = 3k + r, r in {0,1,2};
 * y0 = 2^{-k} 2^{-r/3} (1 - 0.2063 (m - 1)) (chord of m^{-1/3} on [1, 2],
 * within 3 %); four Newton steps take that to a few ulps. */
double oracle_icbrt(double x)
{
    static const double s_r[3] = {1.0, 0.79370052598409973738, 0.62996052494743658238};
    const double third = 1.0 / 3.0;
    uint64_t bits;
    memcpy(&bits, &x, sizeof bits);
    int e = (int)((bits >> 52) & 0x7ff) - 1023;
    uint64_t mb = (bits & 0x000fffffffffffffULL) | 0x3ff0000000000000ULL;
    double m;
    memcpy(&m, &mb, sizeof m);
    int k = (e >= 0) ? e / 3 : -((-e + 2) / 3);
    int r = e - 3 * k;
    uint64_t pb = (uint64_t)(1023 - k) << 52;
    double p2;
    memcpy(&p2, &pb, sizeof p2);
    double y = (1.0 - 0.2063 * (m - 1.0)) * s_r[r] * p2;
    for (int it = 0; it < 4; ++it) {
        double t = x * y * y * y;
        y = y + y * (1.0 - t) * third;
    }
    return y;
}

/* ---------------- grid helpers ---------------- */

static double *alloc_padded(const oracle_t *o)
{
    return (double *)calloc((size_t)o->px * (size_t)o->py, sizeof(double));
}

/* Ghost cells, Sec. 2.2 (boundary conditions through ghost values): two
 * layers per side (second order, Sec. 6.1).  Wall: mirror image with the
 * normal discharge negated.  Outflow: the edge cell is extended. sign = 1
 * for scalars, and the normal component of q gets -1 at walls. */
static void fill_ghost_x(oracle_t *o, double *a, double wall_sign)
{
    int nx = o->nx;
    for (int j = 0; j < o->ny; ++j) {
        for (int k = 0; k < 2; ++k) {
            if (o->p.bc[0] == 0) a[IDX(o, -1 - k, j)] = wall_sign * a[IDX(o, k, j)];
            else                 a[IDX(o, -1 - k, j)] = a[IDX(o, 0, j)];
            if (o->p.bc[1] == 0) a[IDX(o, nx + k, j)] = wall_sign * a[IDX(o, nx - 1 - k, j)];
            else                 a[IDX(o, nx + k, j)] = a[IDX(o, nx - 1, j)];
        }
    }
}

static void fill_ghost_y(oracle_t *o, double *a, double wall_sign)
{
    int ny = o->ny;
    for (int i = 0; i < o->nx; ++i) {
        for (int k = 0; k < 2; ++k) {
            if (o->p.bc[2] == 0) a[IDX(o, i, -1 - k)] = wall_sign * a[IDX(o, i, k)];
            else                 a[IDX(o, i, -1 - k)] = a[IDX(o, i, 0)];
            if (o->p.bc[3] == 0) a[IDX(o, i, ny + k)] = wall_sign * a[IDX(o, i, ny - 1 - k)];
            else                 a[IDX(o, i, ny + k)] = a[IDX(o, i, ny - 1)];
        }
    }
}

/* Speed of the boundary state for an imposed discharge (Sec. 2.2): with
 * c = sqrt(g h), the invariant w - 2c carried out of the domain (w = normal
 * velocity, positive inwards) and w = q / h give q g / c^2 - 2c = R, i.e.
 * p(c) = 2c^3 + R c^2 - q g = 0.  For q g = Q > 0 there is one positive
 * root, p is increasing and convex to its right, and c0 = (max(-R, 0) +
 * (Q/2)^{1/3}) lies to its right; Newton's iteration from there decreases
 * monotonically to it and stops when an update no longer decreases c. */
double oracle_inflow_celerity(double R, double Q)
{
    if (!(Q > 0.0)) return R < 0.0 ? -0.5 * R : 0.0;
    double a = R < 0.0 ? -R : 0.0;
    double x = 0.5 * Q;
    double y = oracle_icbrt(x);             /* x^{-1/3} */
    double c = (a + x * y * y) * 1.0625;    /* above the root */
    for (int it = 0; it < 64; ++it) {
        double p = (2.0 * c + R) * (c * c) - Q;
        double dp = (6.0 * c + 2.0 * R) * c;
        double cn = c - p / dp;
        if (!(cn < c)) break;
        c = cn;
    }
    return c;
}

/* Boundary state of an imposed edge from its edge cell (depth h1, normal
 * discharge qn1 positive inwards, tangential discharge qt1), Sec. 2.2.  The
 * outgoing Riemann invariant R = w1 - 2 sqrt(g h1) is kept; the imposed
 * variable replaces the incoming one. */
void oracle_imposed_state(double g, double h_dry, int type, double hset, double qset,
                          double h1, double qn1, double qt1, double out[3])
{
    double w1 = 0.0, t1 = 0.0;
    if (h1 > h_dry) {
        double r = 1.0 / h1;
        w1 = qn1 * r;
        t1 = qt1 * r;
    }
    double R = w1 - 2.0 * sqrt(g * h1);
    if (type == 4) {                    /* torrential inflow: h and q imposed */
        out[0] = hset; out[1] = qset; out[2] = 0.0;
    } else if (type == 2) {             /* fluvial, h imposed */
        double w = R + 2.0 * sqrt(g * hset);
        out[0] = hset; out[1] = hset * w; out[2] = hset * t1;
    } else {                            /* fluvial, discharge imposed */
        double c = oracle_inflow_celerity(R, qset * g);
        double h = (c * c) / g;
        out[0] = h; out[1] = qset; out[2] = h * t1;
    }
}

static void boundary_conditions(oracle_t *o, double *h, double *qx, double *qy)
{
    fill_ghost_x(o, h, 1.0);
    fill_ghost_x(o, qx, -1.0);
    fill_ghost_x(o, qy, 1.0);
    fill_ghost_y(o, h, 1.0);
    fill_ghost_y(o, qx, 1.0);
    fill_ghost_y(o, qy, -1.0);
    /* imposed edges: both ghost layers hold the boundary state of the edge
     * cell; sides W, E, S, N have inward normals +x, -x, +y, -y */
    for (int side = 0; side < 4; ++side) {
        int type = o->p.bc[side];
        if (type < 2) continue;
        int along = side < 2 ? o->ny : o->nx;
        for (int k = 0; k < along; ++k) {
            int i = side == 0 ? 0 : side == 1 ? o->nx - 1 : k;
            int j = side == 2 ? 0 : side == 3 ? o->ny - 1 : k;
            size_t c = IDX(o, i, j);
            double sgn = (side == 1 || side == 3) ? -1.0 : 1.0;
            double qn = side < 2 ? sgn * qx[c] : sgn * qy[c];
            double qt = side < 2 ? qy[c] : qx[c];
            double b[3];
            oracle_imposed_state(o->p.g, o->p.h_dry, type, o->p.bc_h[side], o->p.bc_q[side],
                                 h[c], qn, qt, b);
            for (int l = 1; l <= 2; ++l) {
                int gi = side == 0 ? -l : side == 1 ? o->nx - 1 + l : i;
                int gj = side == 2 ? -l : side == 3 ? o->ny - 1 + l : j;
                size_t gc = IDX(o, gi, gj);
                h[gc] = b[0];
                if (side < 2) { qx[gc] = sgn * b[1]; qy[gc] = b[2]; }
                else          { qy[gc] = sgn * b[1]; qx[gc] = b[2]; }
            }
        }
    }
}

/* ---------------- the steps of Algorithm 1 ---------------- */

/* Cell velocities u = q/h (one reciprocal of h per cell); zero when dry. */
static void velocities(oracle_t *o, const double *h, const double *qx, const double *qy)
{
    size_t n = (size_t)o->px * (size_t)o->py;
    double hdry = o->p.h_dry;
#pragma omp parallel for schedule(static)
    for (long c = 0; c < (long)n; ++c) {
        if (h[c] > hdry) {
            double rh = 1.0 / h[c];
            o->u[c] = qx[c] * rh;
            o->v[c] = qy[c] * rh;
        } else {
            o->u[c] = 0.0;
            o->v[c] = 0.0;
        }
    }
}

/* MUSCL reconstruction of one cell along one direction (Sec. 3.4), given the
 * cell c and its neighbours cm (minus) and cp (plus).  Reconstructs h,
 * eta = h + z, the normal velocity un and the transverse velocity ut; z is
 * deduced from eta and h; velocities use the discharge-conserving form. */
static void muscl_cell(const oracle_t *o, const double *h, size_t cm, size_t c, size_t cp,
                       const double *un, const double *ut,
                       double *hm, double *hp, double *zm, double *zp,
                       double *unm, double *unp, double *utm, double *utp)
{
    const double *z = o->z;
    double dh = oracle_minmod(h[c] - h[cm], h[cp] - h[c]);
    double hmv = h[c] - 0.5 * dh;
    double hpv = h[c] + 0.5 * dh;
    double em = h[cm] + z[cm], ec = h[c] + z[c], ep = h[cp] + z[cp];
    double de = oracle_minmod(ec - em, ep - ec);
    double etam = ec - 0.5 * de;
    double etap = ec + 0.5 * de;
    *hm = hmv;
    *hp = hpv;
    *zm = etam - hmv;
    *zp = etap - hpv;
    if (h[c] > o->p.h_dry) {
        double rh = 1.0 / h[c];
        double dun = oracle_minmod(un[c] - un[cm], un[cp] - un[c]);
        double dut = oracle_minmod(ut[c] - ut[cm], ut[cp] - ut[c]);
        /* u_{i-1/2+} = u_i - (h_{i+1/2-}/h_i) Du/2, u_{i+1/2-} = u_i + (h_{i-1/2+}/h_i) Du/2 */
        *unm = un[c] - (hpv * rh) * (0.5 * dun);
        *unp = un[c] + (hmv * rh) * (0.5 * dun);
        *utm = ut[c] - (hpv * rh) * (0.5 * dut);
        *utp = ut[c] + (hmv * rh) * (0.5 * dut);
    } else {
        *unm = un[c];
        *unp = un[c];
        *utm = ut[c];
        *utp = ut[c];
    }
}

/* Second order reconstruction over all cells that touch an interior face:
 * x for i in [-1, nx], j in [0, ny); y for i in [0, nx), j in [-1, ny]. */
static void second_order_reconstruction(oracle_t *o, const double *h)
{
    int nx = o->nx, ny = o->ny;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int i = -1; i <= nx; ++i) {
            size_t c = IDX(o, i, j);
            muscl_cell(o, h, IDX(o, i - 1, j), c, IDX(o, i + 1, j), o->u, o->v,
                       &o->xhm[c], &o->xhp[c], &o->xzm[c], &o->xzp[c],
                       &o->xum[c], &o->xup[c], &o->xvm[c], &o->xvp[c]);
        }
#pragma omp parallel for schedule(static)
    for (int j = -1; j <= ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t c = IDX(o, i, j);
            muscl_cell(o, h, IDX(o, i, j - 1), c, IDX(o, i, j + 1), o->v, o->u,
                       &o->yhm[c], &o->yhp[c], &o->yzm[c], &o->yzp[c],
                       &o->yvm[c], &o->yvp[c], &o->yum[c], &o->yup[c]);
        }
}

/* First order (Sec. 3.3, n_CFL = 1): the face values are the cell values,
 * so z_- = z_+ = z_i and the centred term Fc vanishes. */
static void first_order_reconstruction(oracle_t *o, const double *h)
{
    int nx = o->nx, ny = o->ny;
    const double *z = o->z;
#pragma omp parallel for schedule(static)
    for (int j = -1; j <= ny; ++j)
        for (int i = -1; i <= nx; ++i) {
            size_t c = IDX(o, i, j);
            o->xhm[c] = o->xhp[c] = o->yhm[c] = o->yhp[c] = h[c];
            o->xzm[c] = o->xzp[c] = o->yzm[c] = o->yzp[c] = z[c];
            o->xum[c] = o->xup[c] = o->yum[c] = o->yup[c] = o->u[c];
            o->xvm[c] = o->xvp[c] = o->yvm[c] = o->yvp[c] = o->v[c];
        }
}

static void reconstruction(oracle_t *o, const double *h)
{
    if (o->p.order == 1) first_order_reconstruction(o, h);
    else second_order_reconstruction(o, h);
}

/* Hydrostatic reconstruction (Sec. 3.1) + HLL (Sec. 3.3) + the
 * well-balancing corrections S_L, S_R for one face between cell a (left,
 * its plus side) and cell b (right, its minus side). */
static void face_flux(const oracle_t *o,
                      double hpa, double zpa, double unpa, double utpa,
                      double hmb, double zmb, double unmb, double utmb,
                      double *f1, double *f2l, double *f2r, double *f3)
{
    double g = o->p.g;
    double zmax = fmax(zpa, zmb);
    double hL = fmax(0.0, (hpa + zpa) - zmax);
    double hR = fmax(0.0, (hmb + zmb) - zmax);
    double F[3];
    oracle_hll(g, hL, unpa, utpa, hR, unmb, utmb, F);
    *f1 = F[0];
    *f2l = F[1] + 0.5 * g * (hpa * hpa - hL * hL);
    *f2r = F[1] + 0.5 * g * (hmb * hmb - hR * hR);
    *f3 = F[2];
}

static void numerical_flux(oracle_t *o)
{
    int nx = o->nx, ny = o->ny;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int i = -1; i < nx; ++i) {
            size_t a = IDX(o, i, j), b = IDX(o, i + 1, j);
            face_flux(o, o->xhp[a], o->xzp[a], o->xup[a], o->xvp[a],
                      o->xhm[b], o->xzm[b], o->xum[b], o->xvm[b],
                      &o->fx1[a], &o->fx2l[a], &o->fx2r[a], &o->fx3[a]);
        }
#pragma omp parallel for schedule(static)
    for (int j = -1; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t a = IDX(o, i, j), b = IDX(o, i, j + 1);
            face_flux(o, o->yhp[a], o->yzp[a], o->yvp[a], o->yup[a],
                      o->yhm[b], o->yzm[b], o->yvm[b], o->yum[b],
                      &o->fy1[a], &o->fy2l[a], &o->fy2r[a], &o->fy3[a]);
        }
}

/* Scheme computation, Eq. (SW1Dscheme) in x then y, followed by the
 * semi-implicit friction of Sec. 3.2 and the dry clean-up.  Reads the stage
 * input state (h, qx, qy) for U^s and the velocities of U^s. */
static void scheme_and_friction(oracle_t *o, const double *h, const double *qx, const double *qy,
                                double *ho, double *qxo, double *qyo, double dt)
{
    int nx = o->nx, ny = o->ny;
    double g = o->p.g, hdry = o->p.h_dry;
    double dtdx = dt / o->dx, dtdy = dt / o->dy;
    double hg = 0.5 * g;
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t c = IDX(o, i, j), w = IDX(o, i - 1, j), s = IDX(o, i, j - 1);
            /* centred source terms -Fc (Sec. 3.1): g (h_m + h_p)/2 (z_p - z_m) */
            double fcx = hg * (o->xhm[c] + o->xhp[c]) * (o->xzp[c] - o->xzm[c]);
            double fcy = hg * (o->yhm[c] + o->yhp[c]) * (o->yzp[c] - o->yzm[c]);
            double hs = h[c] - dtdx * (o->fx1[c] - o->fx1[w]) - dtdy * (o->fy1[c] - o->fy1[s]);
            double qxs = qx[c] - dtdx * ((o->fx2l[c] - o->fx2r[w]) + fcx)
                               - dtdy * (o->fy3[c] - o->fy3[s]);
            double qys = qy[c] - dtdx * (o->fx3[c] - o->fx3[w])
                               - dtdy * ((o->fy2l[c] - o->fy2r[s]) + fcy);
            if (hs > hdry) {
                if (o->p.friction != 0) {
                    /* q = q* / (1 + dt g C_f |u^s| / h*^p): p = 4/3 for the
                     * Manning-Strickler family, 1 for Darcy-Weisbach-Chezy
                     * (whose g C_f |u| / h is the paper's (f/8)|q|/(h h*)) */
                    double cf = o->cf ? o->cf[(size_t)j * nx + i] : o->p_cf;
                    double speed = sqrt(o->u[c] * o->u[c] + o->v[c] * o->v[c]);
                    double hinv;
                    if (o->p.friction <= 2) {
                        double y = oracle_icbrt(hs);      /* h*^{-1/3} */
                        hinv = (y * y) * (y * y);         /* h*^{-4/3} */
                    } else {
                        hinv = 1.0 / hs;
                    }
                    double den = 1.0 + (dt * g * cf) * speed * hinv;
                    double rden = 1.0 / den;
                    qxs = qxs * rden;
                    qys = qys * rden;
                }
            } else {
                qxs = 0.0;
                qys = 0.0;
            }
            ho[c] = hs;
            qxo[c] = qxs;
            qyo[c] = qys;
        }
}

/* Max over interior cells of |u_face| + sqrt(g h_face) over the MUSCL face
 * values (Eq. (cfl), second order), per direction. */
static void cfl_lambda(const oracle_t *o, double *lx, double *ly)
{
    int nx = o->nx, ny = o->ny;
    double g = o->p.g;
    double ax = 0.0, ay = 0.0;
    int bad = 0;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            size_t c = IDX(o, i, j);
            double a = fmax(fabs(o->xum[c]) + sqrt(g * o->xhm[c]), fabs(o->xup[c]) + sqrt(g * o->xhp[c]));
            double b = fmax(fabs(o->yvm[c]) + sqrt(g * o->yhm[c]), fabs(o->yvp[c]) + sqrt(g * o->yhp[c]));
            if (!isfinite(a) || !isfinite(b)) bad = 1;
            if (a > ax) ax = a;
            if (b > ay) ay = b;
        }
    /* an imposed edge feeds its boundary state into the edge faces' fluxes,
     * so the face value of the first ghost layer facing the domain counts
     * too (both ghost layers are equal, so it is the ghost state itself) */
    for (int j = 0; j < ny; ++j) {
        size_t w = IDX(o, -1, j), e = IDX(o, nx, j);
        if (o->p.bc[0] >= 2) ax = fmax(ax, fabs(o->xup[w]) + sqrt(g * o->xhp[w]));
        if (o->p.bc[1] >= 2) ax = fmax(ax, fabs(o->xum[e]) + sqrt(g * o->xhm[e]));
    }
    for (int i = 0; i < nx; ++i) {
        size_t s = IDX(o, i, -1), n = IDX(o, i, ny);
        if (o->p.bc[2] >= 2) ay = fmax(ay, fabs(o->yvp[s]) + sqrt(g * o->yhp[s]));
        if (o->p.bc[3] >= 2) ay = fmax(ay, fabs(o->yvm[n]) + sqrt(g * o->yhm[n]));
    }
    if (!isfinite(ax) || !isfinite(ay)) bad = 1;
    *lx = bad ? NAN : ax;
    *ly = bad ? NAN : ay;
}

/* Net mass flux out through the domain edges [m^3/s] for the current face
 * fluxes (walls contribute exactly zero). */
static double boundary_outflow(const oracle_t *o)
{
    int nx = o->nx, ny = o->ny;
    double s = 0.0;
    for (int j = 0; j < ny; ++j)
        s += (o->fx1[IDX(o, nx - 1, j)] - o->fx1[IDX(o, -1, j)]) * o->dy;
    for (int i = 0; i < nx; ++i)
        s += (o->fy1[IDX(o, i, ny - 1)] - o->fy1[IDX(o, i, -1)]) * o->dx;
    return s;
}

/* One Heun stage: U_out = U_in + dt Phi(U_in), friction included. */
static double heun_stage(oracle_t *o, double *h, double *qx, double *qy,
                         double *ho, double *qxo, double *qyo, double dt)
{
    boundary_conditions(o, h, qx, qy);
    velocities(o, h, qx, qy);
    reconstruction(o, h);
    numerical_flux(o);
    scheme_and_friction(o, h, qx, qy, ho, qxo, qyo, dt);
    return boundary_outflow(o);
}

/* ---------------- public API ---------------- */

/* Friction factor C_f of Sec. 2.1 from the law's coefficient: Manning n^2,
 * Strickler 1/K^2, Darcy-Weisbach f/(8g), Chezy 1/C^2. */
double oracle_friction_cf(int law, double g, double coef)
{
    switch (law) {
    case 1: return coef * coef;
    case 2: return 1.0 / (coef * coef);
    case 3: return coef / (8.0 * g);
    case 4: return 1.0 / (coef * coef);
    default: return 0.0;
    }
}

oracle_t *oracle_create(int nx, int ny, double dx, double dy, const double *z,
                        const oracle_params *p, const double *n_map, const double *ks_map)
{
    if (nx < 2 || ny < 2 || !(dx > 0) || !(dy > 0) || !z || !p) return NULL;
    oracle_t *o = (oracle_t *)calloc(1, sizeof *o);
    o->nx = nx; o->ny = ny; o->px = nx + 4; o->py = ny + 4;
    o->dx = dx; o->dy = dy; o->p = *p;
    double **pads[] = {&o->z, &o->h, &o->qx, &o->qy, &o->h1, &o->qx1, &o->qy1,
                       &o->h2, &o->qx2, &o->qy2, &o->u, &o->v,
                       &o->xhm, &o->xhp, &o->xzm, &o->xzp, &o->xum, &o->xup, &o->xvm, &o->xvp,
                       &o->yhm, &o->yhp, &o->yzm, &o->yzp, &o->yum, &o->yup, &o->yvm, &o->yvp,
                       &o->fx1, &o->fx2l, &o->fx2r, &o->fx3, &o->fy1, &o->fy2l, &o->fy2r, &o->fy3};
    for (size_t k = 0; k < sizeof pads / sizeof pads[0]; ++k) *pads[k] = alloc_padded(o);
    size_t ni = (size_t)nx * (size_t)ny;
    o->vinf = (double *)calloc(ni, sizeof(double));
    o->p_cf = oracle_friction_cf(p->friction, p->g, p->fric_coef);
    if (n_map) {
        o->cf = (double *)malloc(ni * sizeof(double));
        for (size_t c = 0; c < ni; ++c) o->cf[c] = oracle_friction_cf(p->friction, p->g, n_map[c]);
    }
    if (ks_map) {
        o->ksmap = (double *)malloc(ni * sizeof(double));
        memcpy(o->ksmap, ks_map, ni * sizeof(double));
    }
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) o->z[IDX(o, i, j)] = z[(size_t)j * nx + i];
    fill_ghost_x(o, o->z, 1.0);
    fill_ghost_y(o, o->z, 1.0);
    return o;
}

void oracle_destroy(oracle_t *o)
{
    if (!o) return;
    double *ptrs[] = {o->z, o->h, o->qx, o->qy, o->h1, o->qx1, o->qy1, o->h2, o->qx2, o->qy2,
                      o->u, o->v, o->xhm, o->xhp, o->xzm, o->xzp, o->xum, o->xup, o->xvm, o->xvp,
                      o->yhm, o->yhp, o->yzm, o->yzp, o->yum, o->yup, o->yvm, o->yvp,
                      o->fx1, o->fx2l, o->fx2r, o->fx3, o->fy1, o->fy2l, o->fy2r, o->fy3,
                      o->vinf, o->cf, o->ksmap, o->dt_seq, o->hmax, o->gauge_rec};
    for (size_t k = 0; k < sizeof ptrs / sizeof ptrs[0]; ++k) free(ptrs[k]);
    free(o->gauge_ij);
    free(o);
}

void oracle_set_state(oracle_t *o, const double *h, const double *qx, const double *qy)
{
    for (int j = 0; j < o->ny; ++j)
        for (int i = 0; i < o->nx; ++i) {
            size_t s = (size_t)j * o->nx + i, c = IDX(o, i, j);
            o->h[c] = h[s]; o->qx[c] = qx[s]; o->qy[c] = qy[s];
        }
}

void oracle_get_state(const oracle_t *o, double *h, double *qx, double *qy)
{
    for (int j = 0; j < o->ny; ++j)
        for (int i = 0; i < o->nx; ++i) {
            size_t s = (size_t)j * o->nx + i, c = IDX(o, i, j);
            h[s] = o->h[c]; qx[s] = o->qx[c]; qy[s] = o->qy[c];
        }
}

void oracle_set_vinf(oracle_t *o, const double *v)
{
    memcpy(o->vinf, v, (size_t)o->nx * o->ny * sizeof(double));
}

void oracle_get_vinf(const oracle_t *o, double *v)
{
    memcpy(v, o->vinf, (size_t)o->nx * o->ny * sizeof(double));
}

void oracle_set_time(oracle_t *o, double t) { o->t = t; }

int oracle_set_dt_sequence(oracle_t *o, const double *dts, int n)
{
    free(o->dt_seq);
    o->dt_seq = NULL; o->dt_seq_n = 0; o->dt_seq_pos = 0;
    if (n <= 0 || !dts) return 0;
    o->dt_seq = (double *)malloc((size_t)n * sizeof(double));
    memcpy(o->dt_seq, dts, (size_t)n * sizeof(double));
    o->dt_seq_n = n;
    return 0;
}

/* CFL time step (Eq. (cfl)) from the current U^n, with the clamps. Returns
 * 0, or -7 when a replayed sequence is exhausted, -4 for a non-finite speed,
 * -6 when a fixed dt breaks the CFL bound. *tnext gets the end time. */
static int compute_dt(oracle_t *o, double *dt_out, double *tnext)
{
    double lx, ly;
    boundary_conditions(o, o->h, o->qx, o->qy);
    velocities(o, o->h, o->qx, o->qy);
    reconstruction(o, o->h);
    cfl_lambda(o, &lx, &ly);
    if (!isfinite(lx) || !isfinite(ly)) return -4;
    double t = o->t, dt;
    if (o->dt_seq) {
        if (o->dt_seq_pos >= o->dt_seq_n) return -7;
        dt = o->dt_seq[o->dt_seq_pos++];
        *dt_out = dt;
        *tnext = t + dt;
        return 0;
    }
    if (o->p.dt_fixed > 0.0) {
        dt = o->p.dt_fixed;
        if (dt * (lx / o->dx + ly / o->dy) > o->p.cfl) return -6;
        *dt_out = dt;
        *tnext = t + dt;
        return 0;
    }
    if (o->p.cfl_mode == 0) {
        double den = lx / o->dx + ly / o->dy;
        dt = (den > 0.0) ? o->p.cfl / den : o->p.dt_max;
    } else {
        double a = (lx > 0.0) ? o->dx / lx : INFINITY;
        double b = (ly > 0.0) ? o->dy / ly : INFINITY;
        double m = fmin(a, b);
        dt = isinf(m) ? o->p.dt_max : o->p.cfl * m;
    }
    if (dt > o->p.dt_max) dt = o->p.dt_max;
    double tn = t + dt;
    double ev[3] = {o->p.t_end, o->p.rain_t_on, o->p.rain_t_off};
    int nev = (o->p.rain_rate > 0.0) ? 3 : 1;
    for (int k = 0; k < nev; ++k)
        if (ev[k] > t && ev[k] < t + dt) { dt = ev[k] - t; tn = ev[k]; }
    *dt_out = dt;
    *tnext = tn;
    return 0;
}

/* Advance n Heun steps; dts_out (nullable) receives each step's dt. */
int oracle_step(oracle_t *o, int n, double *dts_out)
{
    int nx = o->nx, ny = o->ny;
    double hdry = o->p.h_dry;
    for (int s = 0; s < n; ++s) {
        double dt, tn;
        int st = compute_dt(o, &dt, &tn);
        if (st) return st;
        /* U* = U^n + dt Phi(U^n); U** = U* + dt Phi(U*) */
        double b1 = heun_stage(o, o->h, o->qx, o->qy, o->h1, o->qx1, o->qy1, dt);
        if (o->p.check_cfl) {
            double lx, ly;
            boundary_conditions(o, o->h1, o->qx1, o->qy1);
            velocities(o, o->h1, o->qx1, o->qy1);
            reconstruction(o, o->h1);
            cfl_lambda(o, &lx, &ly);
            if (dt * (lx / o->dx + ly / o->dy) > o->p.cfl) o->cfl_viol++;
        }
        const int euler = o->p.order == 1;
        if (euler) {
            o->outflow += dt * b1;
        } else {
            double b2 = heun_stage(o, o->h1, o->qx1, o->qy1, o->h2, o->qx2, o->qy2, dt);
            o->outflow += 0.5 * dt * (b1 + b2);
        }
        int rain = o->p.rain_rate > 0.0 && o->t >= o->p.rain_t_on && o->t < o->p.rain_t_off;
        double rdt = dt * o->p.rain_rate;
        double infil = 0.0;
        for (int j = 0; j < ny; ++j) {
            double row_inf = 0.0;
            for (int i = 0; i < nx; ++i) {
                size_t c = IDX(o, i, j), ci = (size_t)j * nx + i;
                /* Heun combine U^{n+1} = (U^n + U**)/2; first order: U* */
                double h, qx, qy;
                if (euler) {
                    h = o->h1[c]; qx = o->qx1[c]; qy = o->qy1[c];
                } else {
                    h = 0.5 * (o->h[c] + o->h2[c]);
                    qx = 0.5 * (o->qx[c] + o->qx2[c]);
                    qy = 0.5 * (o->qy[c] + o->qy2[c]);
                }
                if (rain) h = h + rdt;                      /* explicit rain */
                if (o->p.infiltration) {                    /* Green-Ampt, Sec. 3.5 */
                    double vi = o->vinf[ci];
                    double ks = o->ksmap ? o->ksmap[ci] : o->p.ks;
                    double d;
                    if (vi > 0.0) {
                        double ic = ks * (1.0 + ((o->p.psi + h) * o->p.dtheta) / vi);
                        d = fmin(h, dt * ic);
                    } else {
                        d = h;
                    }
                    h = h - d;
                    o->vinf[ci] = vi + d;
                    row_inf += d;
                }
                if (h <= hdry) { qx = 0.0; qy = 0.0; }
                o->h[c] = h; o->qx[c] = qx; o->qy[c] = qy;
            }
            infil += row_inf;
        }
        if (rain) o->rain_in += rdt * (double)nx * (double)ny * o->dx * o->dy;
        o->infiltrated += infil * o->dx * o->dy;
        o->t = tn;
        o->last_dt = dt;
        o->steps++;
        if (dts_out) dts_out[s] = dt;
        if (o->hmax)
            for (int j = 0; j < ny; ++j)
                for (int i = 0; i < nx; ++i) {
                    size_t ci = (size_t)j * nx + i;
                    o->hmax[ci] = fmax(o->hmax[ci], o->h[IDX(o, i, j)]);
                }
        if (o->n_gauges > 0 && o->gauge_n < o->gauge_cap) {
            double *r = o->gauge_rec + (size_t)o->gauge_n * (size_t)(1 + 3 * o->n_gauges);
            r[0] = o->t;
            for (int g = 0; g < o->n_gauges; ++g) {
                size_t c = IDX(o, o->gauge_ij[2 * g], o->gauge_ij[2 * g + 1]);
                r[1 + 3 * g] = o->h[c];
                r[2 + 3 * g] = o->qx[c];
                r[3 + 3 * g] = o->qy[c];
            }
            o->gauge_n++;
        }
    }
    return 0;
}

/* Running maximum of the depth (flood-extent output): on = 1 starts it
 * from the current state, 0 stops it. */
void oracle_track_max(oracle_t *o, int on)
{
    free(o->hmax);
    o->hmax = NULL;
    if (!on) return;
    o->hmax = (double *)malloc((size_t)o->nx * o->ny * sizeof(double));
    for (int j = 0; j < o->ny; ++j)
        for (int i = 0; i < o->nx; ++i) o->hmax[(size_t)j * o->nx + i] = o->h[IDX(o, i, j)];
}

int oracle_get_max(const oracle_t *o, double *out)
{
    if (!o->hmax) return -10;
    memcpy(out, o->hmax, (size_t)o->nx * o->ny * sizeof(double));
    return 0;
}

/* Gauges at cells (i, j) = ij[2g], ij[2g+1]; up to cap records of
 * t, then (h, qx, qy) per gauge, one after every step. */
int oracle_set_gauges(oracle_t *o, const int *ij, int n, int cap)
{
    free(o->gauge_ij);
    free(o->gauge_rec);
    o->gauge_ij = NULL; o->gauge_rec = NULL;
    o->n_gauges = 0; o->gauge_cap = 0; o->gauge_n = 0;
    if (n <= 0) return 0;
    for (int g = 0; g < n; ++g)
        if (ij[2 * g] < 0 || ij[2 * g] >= o->nx || ij[2 * g + 1] < 0 || ij[2 * g + 1] >= o->ny) return -1;
    o->gauge_ij = (int *)malloc((size_t)2 * n * sizeof(int));
    memcpy(o->gauge_ij, ij, (size_t)2 * n * sizeof(int));
    o->gauge_rec = (double *)calloc((size_t)cap * (1 + 3 * (size_t)n), sizeof(double));
    o->n_gauges = n;
    o->gauge_cap = cap;
    return 0;
}

int oracle_get_gauges(const oracle_t *o, double *out, int max)
{
    int n = o->gauge_n < max ? o->gauge_n : max;
    memcpy(out, o->gauge_rec, (size_t)n * (1 + 3 * (size_t)o->n_gauges) * sizeof(double));
    return n;
}

/* D8 flow direction (Sec. 5.2, the SkelGIS example): for each cell, the
 * neighbour of smallest elevation among those strictly below the cell;
 * code k = 1..8 for the neighbours E, NE, N, NW, W, SW, S, SE (counter-
 * clockwise from +x, rows growing northwards), 0 when no neighbour is
 * lower.  Ties go to the first in that order.  Neighbours outside the grid
 * are not candidates, nor (with use_nodata) those with z <= nodata.
 * Comparisons in float, the type of the DEM. */
void oracle_d8(const float *z, int nx, int ny, int use_nodata, float nodata, unsigned char *dir)
{
    static const int di[8] = {1, 1, 0, -1, -1, -1, 0, 1};
    static const int dj[8] = {0, 1, 1, 1, 0, -1, -1, -1};
#pragma omp parallel for schedule(static)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            float best = z[(size_t)j * nx + i];
            int code = 0;
            for (int k = 0; k < 8; ++k) {
                int a = i + di[k], b = j + dj[k];
                if (a < 0 || a >= nx || b < 0 || b >= ny) continue;
                float v = z[(size_t)b * nx + a];
                if ((!use_nodata || v > nodata) && v < best) {
                    best = v;
                    code = k + 1;
                }
            }
            dir[(size_t)j * nx + i] = (unsigned char)code;
        }
}

/* Pairwise sum (fixed order) of a contiguous array. */
static double pairwise(const double *a, size_t n)
{
    if (n <= 8) {
        double s = 0.0;
        for (size_t k = 0; k < n; ++k) s += a[k];
        return s;
    }
    size_t h = n / 2;
    return pairwise(a, h) + pairwise(a + h, n - h);
}

/* out: t, last_dt, steps, volume, rain_in, infiltrated, outflow, min_h,
 *      cfl_viol, infiltrated depth total */
void oracle_diag(const oracle_t *o, double *out)
{
    int nx = o->nx, ny = o->ny;
    double *rows = (double *)malloc((size_t)ny * sizeof(double));
    double mn = INFINITY;
    for (int j = 0; j < ny; ++j) {
        rows[j] = pairwise(&o->h[IDX(o, 0, j)], (size_t)nx);
        for (int i = 0; i < nx; ++i) mn = fmin(mn, o->h[IDX(o, i, j)]);
    }
    double vol = pairwise(rows, (size_t)ny) * o->dx * o->dy;
    free(rows);
    out[0] = o->t; out[1] = o->last_dt; out[2] = (double)o->steps; out[3] = vol;
    out[4] = o->rain_in; out[5] = o->infiltrated; out[6] = o->outflow; out[7] = mn;
    out[8] = (double)o->cfl_viol;
    out[9] = 0.0;
}

/* CFL speeds of the current state (for tests). */
void oracle_lambda(oracle_t *o, double *lx, double *ly)
{
    boundary_conditions(o, o->h, o->qx, o->qy);
    velocities(o, o->h, o->qx, o->qy);
    reconstruction(o, o->h);
    cfl_lambda(o, lx, ly);
}

int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

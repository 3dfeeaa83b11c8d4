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
 *   (normal discharge negated), outflow extends the edge cell.
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
    int bc[4];             /* W, E, S, N: 0 wall, 1 outflow */
    int friction;          /* 0 none, 1 Manning */
    double manning_n;
    double rain_rate, rain_t_on, rain_t_off;
    int infiltration;
    double ks, psi, dtheta;
    int check_cfl;         /* count dt > CFL bound of U* */
    double dt_fixed;       /* > 0: fixed dt; a CFL violation is an error */
} oracle_params;

typedef struct {
    int nx, ny, px, py;
    double dx, dy;
    oracle_params p;
    double *z, *h, *qx, *qy, *h1, *qx1, *qy1, *h2, *qx2, *qy2;
    double *n2;      /* per-cell n^2 (interior), or NULL */
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

static void boundary_conditions(oracle_t *o, double *h, double *qx, double *qy)
{
    fill_ghost_x(o, h, 1.0);
    fill_ghost_x(o, qx, -1.0);
    fill_ghost_x(o, qy, 1.0);
    fill_ghost_y(o, h, 1.0);
    fill_ghost_y(o, qx, 1.0);
    fill_ghost_y(o, qy, -1.0);
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
                if (o->p.friction == 1) {
                    double n2 = o->n2 ? o->n2[(size_t)j * nx + i] : o->p.manning_n * o->p.manning_n;
                    double speed = sqrt(o->u[c] * o->u[c] + o->v[c] * o->v[c]);
                    double y = oracle_icbrt(hs);          /* h*^{-1/3} */
                    double hinv43 = (y * y) * (y * y);    /* h*^{-4/3} */
                    double den = 1.0 + (dt * g * n2) * speed * hinv43;
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
    second_order_reconstruction(o, h);
    numerical_flux(o);
    scheme_and_friction(o, h, qx, qy, ho, qxo, qyo, dt);
    return boundary_outflow(o);
}

/* ---------------- public API ---------------- */

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
    if (n_map) {
        o->n2 = (double *)malloc(ni * sizeof(double));
        for (size_t c = 0; c < ni; ++c) o->n2[c] = n_map[c] * n_map[c];
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
                      o->vinf, o->n2, o->ksmap, o->dt_seq};
    for (size_t k = 0; k < sizeof ptrs / sizeof ptrs[0]; ++k) free(ptrs[k]);
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
    second_order_reconstruction(o, o->h);
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
            second_order_reconstruction(o, o->h1);
            cfl_lambda(o, &lx, &ly);
            if (dt * (lx / o->dx + ly / o->dy) > o->p.cfl) o->cfl_viol++;
        }
        double b2 = heun_stage(o, o->h1, o->qx1, o->qy1, o->h2, o->qx2, o->qy2, dt);
        o->outflow += 0.5 * dt * (b1 + b2);
        int rain = o->p.rain_rate > 0.0 && o->t >= o->p.rain_t_on && o->t < o->p.rain_t_off;
        double rdt = dt * o->p.rain_rate;
        double infil = 0.0;
        for (int j = 0; j < ny; ++j) {
            double row_inf = 0.0;
            for (int i = 0; i < nx; ++i) {
                size_t c = IDX(o, i, j), ci = (size_t)j * nx + i;
                /* Heun combine U^{n+1} = (U^n + U**)/2 */
                double h = 0.5 * (o->h[c] + o->h2[c]);
                double qx = 0.5 * (o->qx[c] + o->qx2[c]);
                double qy = 0.5 * (o->qy[c] + o->qy2[c]);
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
    }
    return 0;
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
    second_order_reconstruction(o, o->h);
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

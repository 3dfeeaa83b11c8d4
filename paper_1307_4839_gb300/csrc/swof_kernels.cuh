// swof_kernels.cuh -- the stencil kernels of libswof (sm_103a).
//
// One time step (Algorithm 1 of arXiv 1307.4839) is three launches:
//   k_lambda  : wave speeds of U^n on the MUSCL face values (Eq. (cfl)),
//               warp-shuffle + block max, one atomicMax per block on the
//               bits of a non-negative double; the last block computes dt
//               (FP64) and advances the control block.
//   k_stage<1>: U* = U^n + dt Phi(U^n) -- boundary values, MUSCL-minmod
//               (Sec. 3.4), hydrostatic reconstruction + HLL + S_L/S_R/Fc
//               (Sec. 3.1, 3.3), scheme Eq. (SW1Dscheme) in x and y,
//               semi-implicit Manning friction (Sec. 3.2).  Writes U* and
//               its ghost cells.
//   k_stage<2>: the same on U*, then the Heun average with U^n (in place),
//               rain, Green-Ampt (Sec. 3.5), the dry clean-up and ghosts.
// Each CTA owns a BX x BY tile; it stages the tile plus a 2-cell halo of
// (h, q, z) in shared memory, reconstructs every cell that touches one of
// its faces once, computes every face flux once and updates its cells.
//
// FP64 (T = double): every expression follows the oracle's operation order
// and is compiled with -fmad=false, so results match it bit for bit.
// FP32 (T = float): bulk arithmetic in FP32; z enters only as per-face
// differences dz (precomputed in FP64), the hydrostatic reconstruction in
// difference form h_L = max(0, h_- - max(0, z_+ - z_-)), which is the
// paper's formula rearranged and keeps lake-at-rest exact to FP32 rounding
// of h instead of rounding of z.  dt, time and budgets stay FP64.
#pragma once
#include <cuda_runtime.h>

#include <cmath>
#include <type_traits>

#include "swof_internal.h"

namespace swof {

constexpr int BX = 32, BY = 8, NT = BX * BY;
constexpr int AX = BX + 4, AY = BY + 4, SA = AX * AY;   // tile + 2-halo
constexpr int RXW = BX + 2, RXN = RXW * BY;              // x-recon cells
constexpr int RYW = BX, RYN = RYW * (BY + 2);            // y-recon cells
constexpr int FXW = BX + 1, FXN = FXW * BY;              // x faces
constexpr int FYW = BX, FYN = FYW * (BY + 1);            // y faces
constexpr int LX = BX + 2, LY = BY + 2, LA = LX * LY;    // wave-speed tile + 1-halo
constexpr int NW = NT / 32;
constexpr int REDUCE_BLOCKS = 240;

template <typename T>
struct StageSmem {
    T h[SA], za[SA], zb[SA], u[SA], v[SA], rh[SA], qx[SA], qy[SA];
    T xhm[RXN], xhp[RXN], xzm[RXN], xzp[RXN], xum[RXN], xup[RXN], xvm[RXN], xvp[RXN];
    T yhm[RYN], yhp[RYN], yzm[RYN], yzp[RYN], yum[RYN], yup[RYN], yvm[RYN], yvp[RYN];
    T fx1[FXN], fx2l[FXN], fx2r[FXN], fx3[FXN];
    T fy1[FYN], fy2l[FYN], fy2r[FYN], fy3[FYN];
    double red[NW];
    unsigned long long redb[2][NW];
};

__device__ __forceinline__ double mn(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ float mn(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double mx(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float mx(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double ab(double a) { return fabs(a); }
__device__ __forceinline__ float ab(float a) { return fabsf(a); }
__device__ __forceinline__ double sq(double a) { return sqrt(a); }
__device__ __forceinline__ float sq(float a) { return sqrtf(a); }

// minmod limiter (Sec. 3.4)
template <typename T>
__device__ __forceinline__ T minmod(T a, T b)
{
    if (a >= T(0) && b >= T(0)) return mn(a, b);
    if (a <= T(0) && b <= T(0)) return mx(a, b);
    return T(0);
}

// x^{-1/3}: FP64 by Newton's method on y^{-3} - x with a start value from
// the exponent bits (x = m 2^e, e = 3k + r: y0 = 2^-k 2^{-r/3} (1 - 0.2063
// (m - 1))), four steps y <- y + y (1 - x y^3)/3.  FP32 calls rcbrtf.
__device__ __forceinline__ double icbrt(double x)
{
    long long bits = __double_as_longlong(x);
    int e = (int)((bits >> 52) & 0x7ff) - 1023;
    double m = __longlong_as_double((bits & 0x000fffffffffffffLL) | 0x3ff0000000000000LL);
    int k = (e >= 0) ? e / 3 : -((-e + 2) / 3);
    int r = e - 3 * k;
    double p2 = __longlong_as_double((long long)(1023 - k) << 52);
    double sr = (r == 0) ? 1.0 : ((r == 1) ? 0.79370052598409973738 : 0.62996052494743658238);
    double y = (1.0 - 0.2063 * (m - 1.0)) * sr * p2;
    const double third = 1.0 / 3.0;
#pragma unroll
    for (int it = 0; it < 4; ++it) {
        double t = x * y * y * y;
        y = y + y * (1.0 - t) * third;
    }
    return y;
}
__device__ __forceinline__ float icbrt(float x) { return rcbrtf(x); }

template <typename T>
struct Rec {
    T hm, hp, zm, zp, unm, unp, utm, utp;
};

// MUSCL reconstruction of the middle cell of (0, 1, 2) along one direction:
// h, h + z and the velocities (normal un, transverse ut) with the
// discharge-conserving modified form; z deduced from h + z and h.
// FP64: z0..z2 are the cell elevations; zm/zp are absolute.
// FP32: z0 = dz(0->1), z1 = dz(1->2) (z2 unused); zm/zp are relative to z1.
template <typename T>
__device__ __forceinline__ Rec<T> muscl(T h0, T h1, T h2, T z0, T z1, T z2,
                                        T un0, T un1, T un2, T ut0, T ut1, T ut2,
                                        T rh1, T hdry)
{
    Rec<T> r;
    if constexpr (std::is_same<T, double>::value) {
        double dh = minmod(h1 - h0, h2 - h1);
        r.hm = h1 - 0.5 * dh;
        r.hp = h1 + 0.5 * dh;
        double em = h0 + z0, ec = h1 + z1, ep = h2 + z2;
        double de = minmod(ec - em, ep - ec);
        double etam = ec - 0.5 * de;
        double etap = ec + 0.5 * de;
        r.zm = etam - r.hm;
        r.zp = etap - r.hp;
    } else {
        (void)z2;
        float a = h1 - h0, b = h2 - h1;
        float dh = minmod(a, b);
        r.hm = h1 - 0.5f * dh;
        r.hp = h1 + 0.5f * dh;
        float de = minmod(a + z0, b + z1);
        float off = 0.5f * (de - dh);
        r.zm = -off;
        r.zp = off;
    }
    if (h1 > hdry) {
        T dun = minmod(un1 - un0, un2 - un1);
        T dut = minmod(ut1 - ut0, ut2 - ut1);
        r.unm = un1 - (r.hp * rh1) * (T(0.5) * dun);
        r.unp = un1 + (r.hm * rh1) * (T(0.5) * dun);
        r.utm = ut1 - (r.hp * rh1) * (T(0.5) * dut);
        r.utp = ut1 + (r.hm * rh1) * (T(0.5) * dut);
    } else {
        r.unm = un1;
        r.unp = un1;
        r.utm = ut1;
        r.utp = ut1;
    }
    return r;
}

// Max of |u_face| + sqrt(g h_face) over the two MUSCL faces of a cell
// (Eq. (cfl) at second order); only h and the normal velocity are needed.
template <typename T>
__device__ __forceinline__ T cell_speed(T h0, T h1, T h2, T un0, T un1, T un2, T rh1, T hdry, T g)
{
    T dh = minmod(h1 - h0, h2 - h1);
    T hm = h1 - T(0.5) * dh;
    T hp = h1 + T(0.5) * dh;
    T unm = un1, unp = un1;
    if (h1 > hdry) {
        T dun = minmod(un1 - un0, un2 - un1);
        unm = un1 - (hp * rh1) * (T(0.5) * dun);
        unp = un1 + (hm * rh1) * (T(0.5) * dun);
    }
    return mx(ab(unm) + sq(g * hm), ab(unp) + sq(g * hp));
}

// Ordered 64-bit key of a non-negative speed (NaN sorts above everything).
template <typename T>
__device__ __forceinline__ unsigned long long speed_key(T a)
{
    double d = (double)a;
    if (d == 0.0) return 0ull;
    return (unsigned long long)__double_as_longlong(d);
}

// HLL flux (Sec. 3.3) of one face + the well-balancing corrections
// S_L, S_R (Sec. 3.1).  a = left cell's plus side, b = right cell's minus
// side; dz = z_b - z_a (FP32 only).
template <typename T>
__device__ __forceinline__ void face_flux(T g, T hpa, T zpa, T unpa, T utpa,
                                          T hmb, T zmb, T unmb, T utmb, T dz,
                                          T &f1, T &f2l, T &f2r, T &f3)
{
    T hL, hR;
    if constexpr (std::is_same<T, double>::value) {
        (void)dz;
        double zmax = fmax(zpa, zmb);
        hL = fmax(0.0, (hpa + zpa) - zmax);
        hR = fmax(0.0, (hmb + zmb) - zmax);
    } else {
        float zb = dz + zmb;                       // z_+ relative to z_a
        hL = fmaxf(0.0f, hpa - fmaxf(0.0f, zb - zpa));
        hR = fmaxf(0.0f, hmb - fmaxf(0.0f, zpa - zb));
    }
    T F0, F1, F2;
    if (hL == T(0) && hR == T(0)) {
        // both face depths zero: every HLL branch gives exactly zero
        F0 = T(0);
        F1 = T(0);
        F2 = T(0);
    } else {
        T cL = sq(g * hL), cR = sq(g * hR);
        T c1 = mn(unpa - cL, unmb - cR);
        T c2 = mx(unpa + cL, unmb + cR);
        T qL = hL * unpa, qR = hR * unmb;
        T FL0 = qL, FL1 = qL * unpa + T(0.5) * g * hL * hL, FL2 = qL * utpa;
        T FR0 = qR, FR1 = qR * unmb + T(0.5) * g * hR * hR, FR2 = qR * utmb;
        if (c1 >= T(0)) {
            F0 = FL0; F1 = FL1; F2 = FL2;
        } else if (c2 <= T(0)) {
            F0 = FR0; F1 = FR1; F2 = FR2;
        } else {
            T r = T(1) / (c2 - c1);
            T w = c1 * c2 * r;
            F0 = (c2 * FL0 - c1 * FR0) * r + w * (hR - hL);
            F1 = (c2 * FL1 - c1 * FR1) * r + w * (qR - qL);
            F2 = (c2 * FL2 - c1 * FR2) * r + w * (hR * utmb - hL * utpa);
        }
    }
    f1 = F0;
    f2l = F1 + T(0.5) * g * (hpa * hpa - hL * hL);
    f2r = F1 + T(0.5) * g * (hmb * hmb - hR * hR);
    f3 = F2;
}

__device__ __forceinline__ size_t pidx(const Params &P, int gi, int gj)
{
    return (size_t)(gj + 2) * (size_t)P.pitch + (size_t)(gi + P.lpad);
}

// Fixed-order block sum (warp xor tree, then warps in order); thread 0 gets it.
__device__ __forceinline__ double block_sum(double v, double *red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < NW; ++w) s += red[w];
    __syncthreads();
    return s;
}

__device__ __forceinline__ unsigned long long block_max(unsigned long long v, unsigned long long *red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    unsigned long long s = 0;
    if (threadIdx.x == 0)
        for (int w = 0; w < NW; ++w) s = red[w] > s ? red[w] : s;
    __syncthreads();
    return s;
}

// dt of the step (Eq. (cfl), clamps, replay or fixed dt) and the control
// block update.  FP64 throughout; run by one thread of the last block.
template <typename T>
__device__ void control(const Params &P, const Fields<T> &F)
{
    DevCtl *c = F.ctl;
    __threadfence();
    unsigned long long bx = atomicAdd(&c->lam_bits[0], 0ull);
    unsigned long long by = atomicAdd(&c->lam_bits[1], 0ull);
    c->lam_bits[0] = 0ull;
    c->lam_bits[1] = 0ull;
    c->done = 0u;
    double lx = __longlong_as_double((long long)bx);
    double ly = __longlong_as_double((long long)by);
    if (!isfinite(lx) || !isfinite(ly)) {
        c->status = SWOF_ENONFINITE;
        return;
    }
    double t = c->t, dt, tn;
    if (F.dt_seq) {
        if (c->dt_seq_pos >= c->dt_seq_n) {
            c->status = SWOF_EDTSEQ;
            return;
        }
        dt = F.dt_seq[c->dt_seq_pos++];
        tn = t + dt;
    } else if (P.dt_fixed > 0.0) {
        dt = P.dt_fixed;
        if (dt * (lx / P.dx + ly / P.dy) > P.cfl) {
            c->status = SWOF_ECFL;
            return;
        }
        tn = t + dt;
    } else {
        if (P.cfl_mode == SWOF_CFL_SUM) {
            double den = lx / P.dx + ly / P.dy;
            dt = (den > 0.0) ? P.cfl / den : P.dt_max;
        } else {
            double a = (lx > 0.0) ? P.dx / lx : INFINITY;
            double b = (ly > 0.0) ? P.dy / ly : INFINITY;
            double m = fmin(a, b);
            dt = isinf(m) ? P.dt_max : P.cfl * m;
        }
        if (dt > P.dt_max) dt = P.dt_max;
        if (P.dt_min > 0.0 && dt < P.dt_min) {
            c->status = SWOF_EDTUNDERFLOW;
            return;
        }
        tn = t + dt;
        double ev[3] = {P.t_end, P.rain_t_on, P.rain_t_off};
        int nev = (P.rain_rate > 0.0) ? 3 : 1;
        for (int k = 0; k < nev; ++k)
            if (ev[k] > t && ev[k] < t + dt) {
                dt = ev[k] - t;
                tn = ev[k];
            }
    }
    c->dt = dt;
    c->dtdx = dt / P.dx;
    c->dtdy = dt / P.dy;
    int rain = P.rain_rate > 0.0 && t >= P.rain_t_on && t < P.rain_t_off;
    c->rain_active = rain;
    c->rdt = dt * P.rain_rate;
    if (rain) c->rain_in += c->rdt * (double)P.nx * (double)P.ny * P.dx * P.dy;
    if (F.dt_hist && c->steps < F.dt_hist_cap) F.dt_hist[c->steps] = dt;
    c->t = tn;
    c->last_dt = dt;
    c->steps++;
}

// ---------------------------------------------------------------------------
// Wave speeds of U^n and dt.  Grid-stride over BX x BY tiles, 1-cell halo.
template <typename T>
__global__ void __launch_bounds__(NT) k_lambda(Params P, Fields<T> F)
{
    __shared__ T sh[LA], su[LA], sv[LA], srh[LA];
    __shared__ unsigned long long red[2][NW];
    DevCtl *ctl = F.ctl;
    if (ctl->status) return;
    const T hdry = (T)P.h_dry, g = (T)P.g;
    const int tid = threadIdx.x;
    const int tx = (P.nx + BX - 1) / BX, ty = (P.ny + BY - 1) / BY;
    const int ntiles = tx * ty;
    unsigned long long kx = 0ull, ky = 0ull;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int i0 = (tile % tx) * BX, j0 = (tile / tx) * BY;
        for (int idx = tid; idx < LA; idx += NT) {
            int gi = i0 + idx % LX - 1, gj = j0 + idx / LX - 1;
            T h = T(0), qx = T(0), qy = T(0);
            if (gi <= P.nx + 1 && gj <= P.ny + 1) {
                size_t o = pidx(P, gi, gj);
                h = F.h[o];
                qx = F.qx[o];
                qy = F.qy[o];
            }
            T rh = T(0), u = T(0), v = T(0);
            if (h > hdry) {
                rh = T(1) / h;
                u = qx * rh;
                v = qy * rh;
            }
            sh[idx] = h;
            su[idx] = u;
            sv[idx] = v;
            srh[idx] = rh;
        }
        __syncthreads();
        {
            int ti = tid % BX, tj = tid / BX;
            int gi = i0 + ti, gj = j0 + tj;
            if (gi < P.nx && gj < P.ny) {
                int c = (tj + 1) * LX + (ti + 1);
                T ax = cell_speed(sh[c - 1], sh[c], sh[c + 1], su[c - 1], su[c], su[c + 1], srh[c], hdry, g);
                T ay = cell_speed(sh[c - LX], sh[c], sh[c + LX], sv[c - LX], sv[c], sv[c + LX], srh[c], hdry, g);
                unsigned long long a = speed_key(ax), b = speed_key(ay);
                kx = a > kx ? a : kx;
                ky = b > ky ? b : ky;
            }
        }
        __syncthreads();
    }
    kx = block_max(kx, red[0]);
    ky = block_max(ky, red[1]);
    if (tid == 0) {
        atomicMax(&ctl->lam_bits[0], kx);
        atomicMax(&ctl->lam_bits[1], ky);
        __threadfence();
        unsigned int ticket = atomicAdd(&ctl->done, 1u);
        if (ticket == gridDim.x - 1) control(P, F);
    }
}

// ---------------------------------------------------------------------------
// Write one interior cell of a stage output and the ghost cells that mirror
// it (Sec. 2.2: wall = mirror with the normal discharge negated, outflow =
// edge cell extended; two layers).
template <typename T>
__device__ __forceinline__ void store_cell(const Params &P, T *h, T *qx, T *qy, int gi, int gj,
                                           T hv, T qxv, T qyv)
{
    size_t o = pidx(P, gi, gj);
    h[o] = hv;
    qx[o] = qxv;
    qy[o] = qyv;
    if (gi < 2) {            // west
        if (P.bc[0] == SWOF_BC_WALL) {
            size_t g = pidx(P, -1 - gi, gj);
            h[g] = hv; qx[g] = -qxv; qy[g] = qyv;
        } else if (gi == 0) {
            size_t g1 = pidx(P, -1, gj), g2 = pidx(P, -2, gj);
            h[g1] = hv; qx[g1] = qxv; qy[g1] = qyv;
            h[g2] = hv; qx[g2] = qxv; qy[g2] = qyv;
        }
    }
    if (gi >= P.nx - 2) {    // east
        if (P.bc[1] == SWOF_BC_WALL) {
            size_t g = pidx(P, 2 * P.nx - 1 - gi, gj);
            h[g] = hv; qx[g] = -qxv; qy[g] = qyv;
        } else if (gi == P.nx - 1) {
            size_t g1 = pidx(P, P.nx, gj), g2 = pidx(P, P.nx + 1, gj);
            h[g1] = hv; qx[g1] = qxv; qy[g1] = qyv;
            h[g2] = hv; qx[g2] = qxv; qy[g2] = qyv;
        }
    }
    if (gj < 2) {            // south
        if (P.bc[2] == SWOF_BC_WALL) {
            size_t g = pidx(P, gi, -1 - gj);
            h[g] = hv; qx[g] = qxv; qy[g] = -qyv;
        } else if (gj == 0) {
            size_t g1 = pidx(P, gi, -1), g2 = pidx(P, gi, -2);
            h[g1] = hv; qx[g1] = qxv; qy[g1] = qyv;
            h[g2] = hv; qx[g2] = qxv; qy[g2] = qyv;
        }
    }
    if (gj >= P.ny - 2) {    // north
        if (P.bc[3] == SWOF_BC_WALL) {
            size_t g = pidx(P, gi, 2 * P.ny - 1 - gj);
            h[g] = hv; qx[g] = qxv; qy[g] = -qyv;
        } else if (gj == P.ny - 1) {
            size_t g1 = pidx(P, gi, P.ny), g2 = pidx(P, gi, P.ny + 1);
            h[g1] = hv; qx[g1] = qxv; qy[g1] = qyv;
            h[g2] = hv; qx[g2] = qxv; qy[g2] = qyv;
        }
    }
}

// ---------------------------------------------------------------------------
// One Heun stage over a BX x BY tile.
template <typename T, int STAGE>
__global__ void __launch_bounds__(NT) k_stage(Params P, Fields<T> F)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    StageSmem<T> &S = *reinterpret_cast<StageSmem<T> *>(smem_raw);
    const DevCtl *ctl = F.ctl;
    if (ctl->status) return;
    constexpr bool fp64 = std::is_same<T, double>::value;
    const T hdry = (T)P.h_dry, g = (T)P.g;
    const int tid = threadIdx.x;
    const int i0 = blockIdx.x * BX, j0 = blockIdx.y * BY;
    const T *hin = (STAGE == 1) ? F.h : F.h1;
    const T *qxin = (STAGE == 1) ? F.qx : F.qx1;
    const T *qyin = (STAGE == 1) ? F.qy : F.qy1;

    // (A) boundary-filled input tile with halo; velocities u = q/h
    for (int idx = tid; idx < SA; idx += NT) {
        int gi = i0 + idx % AX - 2, gj = j0 + idx / AX - 2;
        T h = T(0), qx = T(0), qy = T(0), za = T(0), zb = T(0);
        if (gi <= P.nx + 1 && gj <= P.ny + 1) {
            size_t o = pidx(P, gi, gj);
            h = hin[o];
            qx = qxin[o];
            qy = qyin[o];
            if constexpr (fp64) {
                za = F.z[o];
            } else {
                za = F.dzx[o];
                zb = F.dzy[o];
            }
        }
        T rh = T(0), u = T(0), v = T(0);
        if (h > hdry) {
            rh = T(1) / h;
            u = qx * rh;
            v = qy * rh;
        }
        S.h[idx] = h; S.za[idx] = za; S.zb[idx] = zb;
        S.u[idx] = u; S.v[idx] = v; S.rh[idx] = rh;
        S.qx[idx] = qx; S.qy[idx] = qy;
    }
    __syncthreads();

    // (B) second-order reconstruction of every cell touching a tile face
    for (int idx = tid; idx < RXN + RYN; idx += NT) {
        if (idx < RXN) {
            int r = idx / RXW, cx = idx % RXW;           // cell (cx - 1, r)
            int c = (r + 2) * AX + (cx + 1);
            Rec<T> q;
            if constexpr (fp64)
                q = muscl<T>(S.h[c - 1], S.h[c], S.h[c + 1], S.za[c - 1], S.za[c], S.za[c + 1],
                             S.u[c - 1], S.u[c], S.u[c + 1], S.v[c - 1], S.v[c], S.v[c + 1], S.rh[c], hdry);
            else
                q = muscl<T>(S.h[c - 1], S.h[c], S.h[c + 1], S.za[c - 1], S.za[c], T(0),
                             S.u[c - 1], S.u[c], S.u[c + 1], S.v[c - 1], S.v[c], S.v[c + 1], S.rh[c], hdry);
            S.xhm[idx] = q.hm; S.xhp[idx] = q.hp; S.xzm[idx] = q.zm; S.xzp[idx] = q.zp;
            S.xum[idx] = q.unm; S.xup[idx] = q.unp; S.xvm[idx] = q.utm; S.xvp[idx] = q.utp;
        } else {
            int k = idx - RXN;
            int r = k / RYW, cx = k % RYW;               // cell (cx, r - 1)
            int c = (r + 1) * AX + (cx + 2);
            Rec<T> q;
            if constexpr (fp64)
                q = muscl<T>(S.h[c - AX], S.h[c], S.h[c + AX], S.za[c - AX], S.za[c], S.za[c + AX],
                             S.v[c - AX], S.v[c], S.v[c + AX], S.u[c - AX], S.u[c], S.u[c + AX], S.rh[c], hdry);
            else
                q = muscl<T>(S.h[c - AX], S.h[c], S.h[c + AX], S.zb[c - AX], S.zb[c], T(0),
                             S.v[c - AX], S.v[c], S.v[c + AX], S.u[c - AX], S.u[c], S.u[c + AX], S.rh[c], hdry);
            S.yhm[k] = q.hm; S.yhp[k] = q.hp; S.yzm[k] = q.zm; S.yzp[k] = q.zp;
            S.yvm[k] = q.unm; S.yvp[k] = q.unp; S.yum[k] = q.utm; S.yup[k] = q.utp;
        }
    }
    __syncthreads();

    // (C) hydrostatic reconstruction + HLL at every face of the tile;
    // boundary faces also feed the outflow budget
    double outacc = 0.0;
    const bool any_out = (P.bc[0] | P.bc[1] | P.bc[2] | P.bc[3]) != 0;
    for (int idx = tid; idx < FXN + FYN; idx += NT) {
        if (idx < FXN) {
            int r = idx / FXW, f = idx % FXW;            // face between (f-1, r) and (f, r)
            int a = r * RXW + f, b = a + 1;
            T dz = T(0);
            if constexpr (!fp64) dz = S.za[(r + 2) * AX + (f + 1)];
            T f1, f2l, f2r, f3;
            face_flux<T>(g, S.xhp[a], S.xzp[a], S.xup[a], S.xvp[a],
                         S.xhm[b], S.xzm[b], S.xum[b], S.xvm[b], dz, f1, f2l, f2r, f3);
            S.fx1[idx] = f1; S.fx2l[idx] = f2l; S.fx2r[idx] = f2r; S.fx3[idx] = f3;
            if (any_out) {
                int gl = i0 + f - 1, gj = j0 + r;
                if (gj < P.ny) {
                    if (gl == -1) outacc -= (double)f1 * P.dy;
                    if (gl == P.nx - 1) outacc += (double)f1 * P.dy;
                }
            }
        } else {
            int k = idx - FXN;
            int f = k / FYW, cx = k % FYW;               // face between (cx, f-1) and (cx, f)
            int a = f * RYW + cx, b = a + RYW;
            T dz = T(0);
            if constexpr (!fp64) dz = S.zb[(f + 1) * AX + (cx + 2)];
            T f1, f2l, f2r, f3;
            face_flux<T>(g, S.yhp[a], S.yzp[a], S.yvp[a], S.yup[a],
                         S.yhm[b], S.yzm[b], S.yvm[b], S.yum[b], dz, f1, f2l, f2r, f3);
            S.fy1[k] = f1; S.fy2l[k] = f2l; S.fy2r[k] = f2r; S.fy3[k] = f3;
            if (any_out) {
                int gl = j0 + f - 1, gi = i0 + cx;
                if (gi < P.nx) {
                    if (gl == -1) outacc -= (double)f1 * P.dx;
                    if (gl == P.ny - 1) outacc += (double)f1 * P.dx;
                }
            }
        }
    }
    __syncthreads();

    // (D) scheme + friction (+ Heun average and sources in stage 2)
    const double dtd = ctl->dt;
    const T dt = (T)dtd, dtdx = (T)ctl->dtdx, dtdy = (T)ctl->dtdy;
    const T hg = T(0.5) * g;
    double infacc = 0.0;
    unsigned long long k2x = 0ull, k2y = 0ull;
    {
        int ti = tid % BX, tj = tid / BX;
        int gi = i0 + ti, gj = j0 + tj;
        if (gi < P.nx && gj < P.ny) {
            int c = (tj + 2) * AX + (ti + 2);
            int rx = tj * RXW + (ti + 1);                // x-recon index of the cell
            int ry = (tj + 1) * RYW + ti;                // y-recon index of the cell
            int fe = tj * FXW + (ti + 1), fw = fe - 1;   // x faces E, W
            int fn = (tj + 1) * FYW + ti, fs = fn - FYW; // y faces N, S
            T fcx = hg * (S.xhm[rx] + S.xhp[rx]) * (S.xzp[rx] - S.xzm[rx]);
            T fcy = hg * (S.yhm[ry] + S.yhp[ry]) * (S.yzp[ry] - S.yzm[ry]);
            T hs = S.h[c] - dtdx * (S.fx1[fe] - S.fx1[fw]) - dtdy * (S.fy1[fn] - S.fy1[fs]);
            T qxs = S.qx[c] - dtdx * ((S.fx2l[fe] - S.fx2r[fw]) + fcx) - dtdy * (S.fy3[fn] - S.fy3[fs]);
            T qys = S.qy[c] - dtdx * (S.fx3[fe] - S.fx3[fw]) - dtdy * ((S.fy2l[fn] - S.fy2r[fs]) + fcy);
            if (hs > hdry) {
                if (P.friction == SWOF_FRIC_MANNING) {
                    size_t o = pidx(P, gi, gj);
                    T n2 = F.n2map ? F.n2map[o] : (T)P.n2;
                    T speed = sq(S.u[c] * S.u[c] + S.v[c] * S.v[c]);
                    T y = icbrt(hs);
                    T hinv43 = (y * y) * (y * y);
                    T den = T(1) + (dt * g * n2) * speed * hinv43;
                    T rden = T(1) / den;
                    qxs = qxs * rden;
                    qys = qys * rden;
                }
            } else {
                qxs = T(0);
                qys = T(0);
            }
            if (STAGE == 1) {
                store_cell<T>(P, F.h1, F.qx1, F.qy1, gi, gj, hs, qxs, qys);
            } else {
                if (P.check_cfl) {
                    T sx = mx(ab(S.xum[rx]) + sq(g * S.xhm[rx]), ab(S.xup[rx]) + sq(g * S.xhp[rx]));
                    T sy = mx(ab(S.yvm[ry]) + sq(g * S.yhm[ry]), ab(S.yvp[ry]) + sq(g * S.yhp[ry]));
                    k2x = speed_key(sx);
                    k2y = speed_key(sy);
                }
                size_t o = pidx(P, gi, gj);
                T h = T(0.5) * (F.h[o] + hs);
                T qx = T(0.5) * (F.qx[o] + qxs);
                T qy = T(0.5) * (F.qy[o] + qys);
                if (ctl->rain_active) h = h + (T)ctl->rdt;
                if (P.infiltration) {
                    T vi = F.vinf[o];
                    T ks = F.ksmap ? F.ksmap[o] : (T)P.ks;
                    T d;
                    if (vi > T(0)) {
                        T ic = ks * (T(1) + (((T)P.psi + h) * (T)P.dtheta) / vi);
                        d = mn(h, dt * ic);
                    } else {
                        d = h;
                    }
                    h = h - d;
                    F.vinf[o] = vi + d;
                    infacc = (double)d;
                }
                if (h <= hdry) {
                    qx = T(0);
                    qy = T(0);
                }
                store_cell<T>(P, F.h, F.qx, F.qy, gi, gj, h, qx, qy);
            }
        }
    }

    // per-block FP64 budget slots (fixed order: deterministic)
    const int blk = blockIdx.y * gridDim.x + blockIdx.x;
    if (any_out) {
        double s = block_sum(outacc, S.red);
        if (tid == 0) F.outflow_slots[blk] += 0.5 * dtd * s;
    }
    if (STAGE == 2 && P.infiltration) {
        double s = block_sum(infacc, S.red);
        if (tid == 0) F.infil_slots[blk] += s;
    }
    if (STAGE == 2 && P.check_cfl) {
        k2x = block_max(k2x, S.redb[0]);
        k2y = block_max(k2y, S.redb[1]);
        if (tid == 0) {
            DevCtl *c = F.ctl;
            atomicMax(&c->lam2_bits[0], k2x);
            atomicMax(&c->lam2_bits[1], k2y);
            __threadfence();
            unsigned int nb = gridDim.x * gridDim.y;
            if (atomicAdd(&c->done2, 1u) == nb - 1) {
                __threadfence();
                double lx = __longlong_as_double((long long)atomicAdd(&c->lam2_bits[0], 0ull));
                double ly = __longlong_as_double((long long)atomicAdd(&c->lam2_bits[1], 0ull));
                c->lam2_bits[0] = 0ull;
                c->lam2_bits[1] = 0ull;
                c->done2 = 0u;
                if (dtd * (lx / P.dx + ly / P.dy) > P.cfl) c->cfl_viol++;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Ghost cells of U^n from its interior (used after a state is set).
template <typename T>
__global__ void k_ghosts(Params P, Fields<T> F)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < P.ny) {
        int gj = k;
        for (int s = 0; s < 2; ++s) {
            int gi = (s == 0) ? 0 : P.nx - 1;
            for (int l = 0; l < 2; ++l) {
                int src = (s == 0) ? l : P.nx - 1 - l;
                int dst = (s == 0) ? -1 - l : P.nx + l;
                int b = P.bc[s];
                int from = (b == SWOF_BC_WALL) ? src : gi;
                T sign = (b == SWOF_BC_WALL) ? T(-1) : T(1);
                size_t o = pidx(P, from, gj), d = pidx(P, dst, gj);
                F.h[d] = F.h[o];
                F.qx[d] = sign * F.qx[o];
                F.qy[d] = F.qy[o];
            }
        }
    } else if (k < P.ny + P.nx) {
        int gi = k - P.ny;
        for (int s = 0; s < 2; ++s) {
            int gj = (s == 0) ? 0 : P.ny - 1;
            for (int l = 0; l < 2; ++l) {
                int src = (s == 0) ? l : P.ny - 1 - l;
                int dst = (s == 0) ? -1 - l : P.ny + l;
                int b = P.bc[2 + s];
                int from = (b == SWOF_BC_WALL) ? src : gj;
                T sign = (b == SWOF_BC_WALL) ? T(-1) : T(1);
                size_t o = pidx(P, gi, from), d = pidx(P, gi, dst);
                F.h[d] = F.h[o];
                F.qx[d] = F.qx[o];
                F.qy[d] = sign * F.qy[o];
            }
        }
    }
}

// Deterministic partial reductions for the diagnostics: per block, the sum
// and min of interior h and the sums of the budget slots, in fixed order.
// out[4*b + 0..3] = sum h, min h, sum outflow slots, sum infiltration slots.
template <typename T>
__global__ void __launch_bounds__(NT) k_reduce(Params P, Fields<T> F, double *out, int nslots)
{
    __shared__ double red[NW];
    __shared__ double redm[NW];
    double s = 0.0, m = INFINITY, so = 0.0, si = 0.0;
    for (int gj = blockIdx.x; gj < P.ny; gj += gridDim.x)
        for (int gi = threadIdx.x; gi < P.nx; gi += NT) {
            double h = (double)F.h[pidx(P, gi, gj)];
            s += h;
            m = fmin(m, h);
        }
    for (int k = blockIdx.x * NT + threadIdx.x; k < nslots; k += gridDim.x * NT) {
        so += F.outflow_slots[k];
        si += F.infil_slots[k];
    }
    s = block_sum(s, red);
    so = block_sum(so, red);
    si = block_sum(si, red);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) redm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double mm = INFINITY;
        for (int w = 0; w < NW; ++w) mm = fmin(mm, redm[w]);
        out[4 * blockIdx.x + 0] = s;
        out[4 * blockIdx.x + 1] = mm;
        out[4 * blockIdx.x + 2] = so;
        out[4 * blockIdx.x + 3] = si;
    }
}

// ---------------------------------------------------------------------------
// Launchers
template <typename T>
int launch_ghosts_t(const Params &P, void *f, void *stream)
{
    const Fields<T> &F = *static_cast<const Fields<T> *>(f);
    int n = P.nx + P.ny;
    k_ghosts<T><<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(P, F);
    return (int)cudaGetLastError();
}

inline int lambda_grid(const Params &P)
{
    int tiles = ((P.nx + BX - 1) / BX) * ((P.ny + BY - 1) / BY);
    int cap = 152 * 8;
    return tiles < cap ? tiles : cap;
}

template <typename T>
int launch_lambda_t(const Params &P, void *f, void *stream)
{
    const Fields<T> &F = *static_cast<const Fields<T> *>(f);
    k_lambda<T><<<lambda_grid(P), NT, 0, (cudaStream_t)stream>>>(P, F);
    return (int)cudaGetLastError();
}

template <typename T>
int configure_t()
{
    int smem = (int)sizeof(StageSmem<T>);
    cudaError_t e = cudaFuncSetAttribute(k_stage<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_stage<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    return (int)e;
}

template <typename T, int STAGE>
int launch_stage_t(const Params &P, void *f, void *stream)
{
    const Fields<T> &F = *static_cast<const Fields<T> *>(f);
    size_t smem = sizeof(StageSmem<T>);
    dim3 grid((P.nx + BX - 1) / BX, (P.ny + BY - 1) / BY);
    k_stage<T, STAGE><<<grid, NT, smem, (cudaStream_t)stream>>>(P, F);
    return (int)cudaGetLastError();
}

template <typename T>
int launch_reduce_t(const Params &P, void *f, double *out, int nslots, void *stream)
{
    const Fields<T> &F = *static_cast<const Fields<T> *>(f);
    k_reduce<T><<<REDUCE_BLOCKS, NT, 0, (cudaStream_t)stream>>>(P, F, out, nslots);
    return (int)cudaGetLastError();
}

// Dense [ny][nx] arrays of type S <-> the padded state of type T.
template <typename T, typename S>
__global__ void k_unpack(Params P, Fields<T> F, const S *h, const S *qx, const S *qy)
{
    size_t n = (size_t)P.nx * P.ny;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        int gi = (int)(k % P.nx), gj = (int)(k / P.nx);
        size_t o = pidx(P, gi, gj);
        F.h[o] = (T)h[k];
        F.qx[o] = (T)qx[k];
        F.qy[o] = (T)qy[k];
    }
}

template <typename T, typename S>
__global__ void k_pack(Params P, Fields<T> F, S *h, S *qx, S *qy)
{
    size_t n = (size_t)P.nx * P.ny;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
        int gi = (int)(k % P.nx), gj = (int)(k / P.nx);
        size_t o = pidx(P, gi, gj);
        h[k] = (S)F.h[o];
        qx[k] = (S)F.qx[o];
        qy[k] = (S)F.qy[o];
    }
}

template <typename T>
int launch_unpack_t(const Params &P, void *f, const void *h, const void *qx, const void *qy,
                    int dtype, void *stream)
{
    const Fields<T> &F = *static_cast<const Fields<T> *>(f);
    cudaStream_t s = (cudaStream_t)stream;
    if (dtype == SWOF_FP64)
        k_unpack<T, double><<<1216, 256, 0, s>>>(P, F, (const double *)h, (const double *)qx, (const double *)qy);
    else
        k_unpack<T, float><<<1216, 256, 0, s>>>(P, F, (const float *)h, (const float *)qx, (const float *)qy);
    return (int)cudaGetLastError();
}

template <typename T>
int launch_pack_t(const Params &P, void *f, void *h, void *qx, void *qy, int dtype, void *stream)
{
    const Fields<T> &F = *static_cast<const Fields<T> *>(f);
    cudaStream_t s = (cudaStream_t)stream;
    if (dtype == SWOF_FP64)
        k_pack<T, double><<<1216, 256, 0, s>>>(P, F, (double *)h, (double *)qx, (double *)qy);
    else
        k_pack<T, float><<<1216, 256, 0, s>>>(P, F, (float *)h, (float *)qx, (float *)qy);
    return (int)cudaGetLastError();
}

inline int stage_slots(const Params &P)
{
    return ((P.nx + BX - 1) / BX) * ((P.ny + BY - 1) / BY);
}

}  // namespace swof

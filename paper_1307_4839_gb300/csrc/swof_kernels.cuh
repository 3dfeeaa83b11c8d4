// swof_kernels.cuh -- the stencil kernels of libswof (sm_103a).
//
// One time step (Algorithm 1 of arXiv 1307.4839) is three launches:
//   k_lambda  : wave speeds of U^n on the MUSCL face values (Eq. (cfl)),
//               warp-shuffle + block max, one atomicMax per block on the
//               bits of a non-negative double; the last block computes dt
//               (FP64) and advances the control block.
//   k_sweep<1>: U* = U^n + dt Phi(U^n) -- boundary values, MUSCL-minmod
//               (Sec. 3.4), hydrostatic reconstruction + HLL + S_L/S_R/Fc
//               (Sec. 3.1, 3.3), scheme Eq. (SW1Dscheme) in x and y,
//               semi-implicit Manning friction (Sec. 3.2).  Writes U* and
//               its ghost cells.
//   k_sweep<2>: the same on U*, then the Heun average with U^n (in place),
//               rain, Green-Ampt (Sec. 3.5), the dry clean-up and ghosts.
// The stage kernels walk columns down the grid (swof_sweep.cuh): every cell
// is reconstructed once per direction, every face flux computed once.
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

constexpr int BX = 32, BY = 8, NT = BX * BY;              // wave-speed kernel tile
constexpr int LX = BX + 2, LY = BY + 2, LA = LX * LY;    // wave-speed tile + 1-halo
constexpr int NW = NT / 32;
constexpr int REDUCE_BLOCKS = 240;

// 4-vectors for shared memory: one 128-bit (FP32) or 2 x 128-bit (FP64)
// access per 4 values.
template <typename T>
struct alignas(4 * sizeof(T)) V4 {
    T x, y, z, w;
};
template <typename T>
struct alignas(2 * sizeof(T)) V2 {
    T x, y;
};

__device__ __forceinline__ double mn(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ float mn(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double mx(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float mx(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double ab(double a) { return fabs(a); }
__device__ __forceinline__ float ab(float a) { return fabsf(a); }
// FP64: IEEE square root and division (the oracle's).  FP32: the PTX
// approximate forms (sqrt.approx: relative error ~2^-23, sqrt(+0) = +0;
// rcp.approx: 1 ulp), never applied to a zero divisor.
__device__ __forceinline__ double sq(double a) { return sqrt(a); }
__device__ __forceinline__ float sq(float a)
{
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}
__device__ __forceinline__ double rcp(double a) { return 1.0 / a; }
__device__ __forceinline__ float rcp(float a)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}

// Scalar parameters in the kernel's precision (no conversions on the path).
template <typename T>
struct Scal {
    T g, hdry, n2, psi, dtheta, ks;
};
template <typename T>
__device__ __forceinline__ Scal<T> scal(const Params &P)
{
    if constexpr (std::is_same<T, double>::value)
        return {P.g, P.h_dry, P.n2, P.psi, P.dtheta, P.ks};
    else
        return {P.fg, P.fh_dry, P.fn2, P.fpsi, P.fdtheta, P.fks};
}

// minmod limiter (Sec. 3.4): the value of smaller magnitude when a and b
// have the same sign, else 0.
//  FP64: decided on the IEEE bit patterns with integer operations (sign bits
//  differ -> 0, else the smaller magnitude); this returns exactly the value
//  of the comparison-based definition (up to the sign of a zero result) and
//  keeps the work off GB300's narrow FP64 pipe.
//  FP32: the same on 32-bit patterns.
__device__ __forceinline__ double minmod(double a, double b)
{
    long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
    if ((ia ^ ib) < 0) return 0.0;
    long long ma = ia & 0x7fffffffffffffffLL, mb = ib & 0x7fffffffffffffffLL;
    return ma <= mb ? a : b;
}
__device__ __forceinline__ float minmod(float a, float b)
{
    int ia = __float_as_int(a), ib = __float_as_int(b);
    if ((ia ^ ib) < 0) return 0.0f;
    int ma = ia & 0x7fffffff, mb = ib & 0x7fffffff;
    return ma <= mb ? a : b;
}

// max(0, x) (the hydrostatic cut, Sec. 3.1); FP64 by the sign bit.
__device__ __forceinline__ double pos(double x)
{
    return (__double_as_longlong(x) < 0) ? 0.0 : x;
}
__device__ __forceinline__ float pos(float x) { return fmaxf(0.0f, x); }

// max / min of two doubles through order-preserving integer keys (same value
// as fmax / fmin for finite inputs, again off the FP64 pipe).
__device__ __forceinline__ long long okey(double x)
{
    long long i = __double_as_longlong(x);
    return i ^ ((i >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double dmax(double a, double b) { return okey(a) >= okey(b) ? a : b; }
__device__ __forceinline__ double dmin(double a, double b) { return okey(a) <= okey(b) ? a : b; }
__device__ __forceinline__ float dmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ float dmin(float a, float b) { return fminf(a, b); }

// x^{-1/3}: FP64 by Newton's method on y^{-3} - x with a start value from
// the exponent bits (x = m 2^e, e = 3k + r: y0 = 2^-k 2^{-r/3} (1 - 0.2063
// (m - 1))), four steps y <- y + y (1 - x y^3)/3.  FP32: 2^{-log2(x)/3} (PTX approximations).
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
__device__ __forceinline__ float icbrt(float x)
{
    // x^{-1/3} = 2^{-log2(x)/3} with the PTX approximate log2 / exp2
    float l, r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l) : "f"(x));
    l = l * (-1.0f / 3.0f);
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(l));
    return r;
}

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

// Ordered key of a non-negative speed: the bits of the value (NaN sorts
// above everything, -0 maps to 0).  FP32 keys are 32-bit so the FP32 path
// needs no FP64 instruction per cell; key64() widens one winner per block.
__device__ __forceinline__ unsigned long long speed_key(double a)
{
    unsigned long long k = (unsigned long long)__double_as_longlong(a);
    return (k == 0x8000000000000000ull) ? 0ull : k;
}
__device__ __forceinline__ unsigned int speed_key(float a)
{
    unsigned int k = __float_as_uint(a);
    return (k == 0x80000000u) ? 0u : k;
}
__device__ __forceinline__ unsigned long long key64(unsigned long long k) { return k; }
__device__ __forceinline__ unsigned long long key64(unsigned int k)
{
    float f = __uint_as_float(k);
    return k == 0u ? 0ull : (unsigned long long)__double_as_longlong((double)f);
}
template <typename K>
__device__ __forceinline__ K kmax(K a, K b) { return a > b ? a : b; }

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
        double zmax = dmax(zpa, zmb);
        hL = pos((hpa + zpa) - zmax);
        hR = pos((hmb + zmb) - zmax);
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
        T c1 = dmin(unpa - cL, unmb - cR);
        T c2 = dmax(unpa + cL, unmb + cR);
        T qL = hL * unpa, qR = hR * unmb;
        T FL0 = qL, FL1 = qL * unpa + T(0.5) * g * hL * hL, FL2 = qL * utpa;
        T FR0 = qR, FR1 = qR * unmb + T(0.5) * g * hR * hR, FR2 = qR * utmb;
        if (c1 >= T(0)) {
            F0 = FL0; F1 = FL1; F2 = FL2;
        } else if (c2 <= T(0)) {
            F0 = FR0; F1 = FR1; F2 = FR2;
        } else {
            T r = rcp(c2 - c1);
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

template <typename K>
__device__ __forceinline__ K block_max(K v, K *red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = kmax(v, (K)__shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    K s = 0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s = kmax(s, red[w]);
    __syncthreads();
    return s;
}

// Sum of one value per thread of T, returned in FP64 to thread 0: FP32 warps
// reduce in FP32 and widen one value per warp (fixed order throughout).
template <typename T>
__device__ __forceinline__ double block_sum_t(T v, double *red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
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
    c->fdt = (float)c->dt;
    c->fdtdx = (float)c->dtdx;
    c->fdtdy = (float)c->dtdy;
    c->frdt = (float)c->rdt;
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
    using K = decltype(speed_key(T(0)));
    __shared__ V4<T> st[LA];   // {h, u, v, 1/h}
    __shared__ K red[2][NW];
    DevCtl *ctl = F.ctl;
    if (ctl->status) return;
    const Scal<T> C = scal<T>(P);
    const int tid = threadIdx.x;
    const int tx = (P.nx + BX - 1) / BX, ty = (P.ny + BY - 1) / BY;
    const int ntiles = tx * ty;
    K kx = 0, ky = 0;
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
            V4<T> e = {h, T(0), T(0), T(0)};
            if (h > C.hdry) {
                e.w = rcp(h);
                e.y = qx * e.w;
                e.z = qy * e.w;
            }
            st[idx] = e;
        }
        __syncthreads();
        {
            int ti = tid % BX, tj = tid / BX;
            int gi = i0 + ti, gj = j0 + tj;
            if (gi < P.nx && gj < P.ny) {
                int c = (tj + 1) * LX + (ti + 1);
                V4<T> m = st[c], w = st[c - 1], e = st[c + 1], s_ = st[c - LX], n = st[c + LX];
                T ax = cell_speed(w.x, m.x, e.x, w.y, m.y, e.y, m.w, C.hdry, C.g);
                T ay = cell_speed(s_.x, m.x, n.x, s_.z, m.z, n.z, m.w, C.hdry, C.g);
                kx = kmax(kx, speed_key(ax));
                ky = kmax(ky, speed_key(ay));
            }
        }
        __syncthreads();
    }
    kx = block_max(kx, red[0]);
    ky = block_max(ky, red[1]);
    if (tid == 0) {
        atomicMax(&ctl->lam_bits[0], key64(kx));
        atomicMax(&ctl->lam_bits[1], key64(ky));
        if (P.lam_partial) return;
        __threadfence();
        unsigned int ticket = atomicAdd(&ctl->done, 1u);
        if (ticket == gridDim.x - 1) control(P, F);
    }
}

// ---------------------------------------------------------------------------
// Wave speeds of U^n on the tile-edge columns and rows the fused stage-2
// kernel of the previous step left out (x speeds on ring columns, y speeds
// on ring rows, read back from the stored U^n and its ghosts), merged into
// the same reduction words; the last block computes dt.
template <typename T>
__device__ __forceinline__ V4<T> cell_rec(const Params &P, const Fields<T> &F, int gi, int gj, T hdry)
{
    size_t o = pidx(P, gi, gj);
    T h = F.h[o];
    V4<T> e = {h, T(0), T(0), T(0)};
    if (h > hdry) {
        e.w = rcp(h);
        e.y = F.qx[o] * e.w;
        e.z = F.qy[o] * e.w;
    }
    return e;
}

template <typename T>
__global__ void __launch_bounds__(NT) k_lambda_ring(Params P, Fields<T> F)
{
    using K = decltype(speed_key(T(0)));
    __shared__ K red[2][NW];
    DevCtl *ctl = F.ctl;
    if (ctl->status) return;
    const Scal<T> C = scal<T>(P);
    K kx = 0, ky = 0;
    const long long nxr = (long long)F.n_ring_cols * P.ny;
    const long long total = nxr + (long long)F.n_ring_rows * P.nx;
    for (long long k = blockIdx.x * (long long)NT + threadIdx.x; k < total; k += (long long)gridDim.x * NT) {
        if (k < nxr) {
            int gj = (int)(k / F.n_ring_cols), gi = F.ring_cols[k % F.n_ring_cols];
            V4<T> w = cell_rec(P, F, gi - 1, gj, C.hdry), m = cell_rec(P, F, gi, gj, C.hdry),
                  e = cell_rec(P, F, gi + 1, gj, C.hdry);
            kx = kmax(kx, speed_key(cell_speed(w.x, m.x, e.x, w.y, m.y, e.y, m.w, C.hdry, C.g)));
        } else {
            long long q = k - nxr;
            int gj = F.ring_rows[q / P.nx], gi = (int)(q % P.nx);
            V4<T> s_ = cell_rec(P, F, gi, gj - 1, C.hdry), m = cell_rec(P, F, gi, gj, C.hdry),
                  n = cell_rec(P, F, gi, gj + 1, C.hdry);
            ky = kmax(ky, speed_key(cell_speed(s_.x, m.x, n.x, s_.z, m.z, n.z, m.w, C.hdry, C.g)));
        }
    }
    kx = block_max(kx, red[0]);
    ky = block_max(ky, red[1]);
    if (threadIdx.x == 0) {
        atomicMax(&ctl->lam_bits[0], key64(kx));
        atomicMax(&ctl->lam_bits[1], key64(ky));
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

}  // namespace swof
#include "swof_sweep.cuh"
namespace swof {

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
int launch_lambda_ring_t(const Params &P, void *f, void *stream)
{
    const Fields<T> &F = *static_cast<const Fields<T> *>(f);
    long long total = (long long)F.n_ring_cols * P.ny + (long long)F.n_ring_rows * P.nx;
    long long b = (total + NT - 1) / NT;
    int grid = (int)(b < 152 * 8 ? (b > 0 ? b : 1) : 152 * 8);
    k_lambda_ring<T><<<grid, NT, 0, (cudaStream_t)stream>>>(P, F);
    return (int)cudaGetLastError();
}

template <typename T>
int configure_t()
{
    return (int)cudaSuccess;
}

template <typename T, int STAGE, int NTX, int H>
int launch_sweep(const Params &P, const Fields<T> &F, cudaStream_t s)
{
    dim3 grid((P.nx + NTX - 5) / (NTX - 4), (P.ny + H - 1) / H);
    k_sweep<T, STAGE, NTX, H><<<grid, NTX, 0, s>>>(P, F);
    return (int)cudaGetLastError();
}

template <typename T, int STAGE>
int launch_stage_t(const Params &P, void *f, void *stream)
{
    const Fields<T> &F = *static_cast<const Fields<T> *>(f);
    cudaStream_t s = (cudaStream_t)stream;
    switch (STAGE == 1 ? P.tile_cfg : P.tile_cfg2) {
    case 1: return launch_sweep<T, STAGE, 128, 64>(P, F, s);
    case 2: return launch_sweep<T, STAGE, 256, 32>(P, F, s);
    case 3: return launch_sweep<T, STAGE, 64, 64>(P, F, s);
    default: return launch_sweep<T, STAGE, 128, 32>(P, F, s);
    }
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

inline int stage_slots(const Params &P) { return max_stage_blocks(P.nx, P.ny); }

}  // namespace swof

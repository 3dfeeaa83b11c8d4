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
//               semi-implicit friction (Sec. 3.2, the laws of Sec. 2.1).
//               Writes U* and its ghost cells (imposed edges: the boundary
//               state of Sec. 2.2).
//   k_sweep<2>: the same on U*, then the Heun average with U^n (in place),
//               rain, Green-Ampt (Sec. 3.5), the dry clean-up and ghosts,
//               and the wave speeds of U^{n+1} inside its tile; the next
//               step's first launch (k_lambda_ring) adds the tile edges.
// The stage kernels walk columns down the grid (swof_sweep.cuh): every cell
// is reconstructed once per direction, every face flux computed once.  The
// first-order step (Sec. 3.3) is the stage with face values = cell values
// followed by k_commit1 (sources, ghosts, speeds).
//
// FP64 (T = double): every expression follows the oracle's operation order
// and is compiled with -fmad=false, so results match it bit for bit; where a
// dry cell's result is known exactly (+0 fluxes, +0 state) the arithmetic
// that would produce it is skipped.
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
#include "tc05.cuh"

SWOF_KERNELS_BEGIN

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
// approximate square root (sqrt.approx: relative error ~2^-23, sqrt(+0) =
// +0) and a reciprocal within an ulp of 1/a: rcp.approx refined by one
// Newton-Raphson step r + r (1 - a r) (never applied to a zero divisor).  The
// reciprocal feeds every velocity u = q (1/h); measured on the 4096^2 valley
// after 2000 steps, a reciprocal of this accuracy halves the FP32 path's
// error against FP64 compared with rcp.approx alone (h 2.1e-6 -> 0.9e-6, hu
// 2.3e-5 -> 1.3e-5, hv 8.6e-6 -> 3.8e-6 relative L1); the errors were the
// same as with the correctly rounded rcp.rn to the last digit on every
// workload, at ~10 % less time on a wet grid; a rounded square root added
// nothing measurable.
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
    return fmaf(r, fmaf(-a, r, 1.0f), r);    // one Newton-Raphson step: within an ulp of 1/a
}

// Scalar parameters in the kernel's precision (no conversions on the path).
template <typename T>
struct Scal {
    T g, hdry, cf, psi, dtheta, ks;
};
template <typename T>
__device__ __forceinline__ Scal<T> scal(const Params &P)
{
    if constexpr (std::is_same<T, double>::value)
        return {P.g, P.h_dry, P.cf, P.psi, P.dtheta, P.ks};
    else
        return {P.fg, P.fh_dry, P.fcf, P.fpsi, P.fdtheta, P.fks};
}

// x == 0 of either sign; FP64 on the bit pattern, off GB300's narrow FP64
// pipe (same answer as the comparison, NaN included).
__device__ __forceinline__ bool is0(double x) { return (__double_as_longlong(x) << 1) == 0; }
__device__ __forceinline__ bool is0(float x) { return x == 0.0f; }

// x > c and x <= c for a threshold c >= +0 (the dry depth): FP64 on the
// bit patterns, which order like the values for non-negative doubles, with
// negative x (sign bit set) below c and NaN on neither side -- the same
// answer as the comparison for every x.
__device__ __forceinline__ bool gt_pos(double x, double c)
{
    const long long b = __double_as_longlong(x);
    return b > __double_as_longlong(c) && b <= 0x7ff0000000000000LL;
}
__device__ __forceinline__ bool le_pos(double x, double c)
{
    const long long b = __double_as_longlong(x);
    const bool nan = (b & 0x7fffffffffffffffLL) > 0x7ff0000000000000LL;
    return !nan && b <= __double_as_longlong(c);
}
__device__ __forceinline__ bool gt_pos(float x, float c) { return x > c; }
__device__ __forceinline__ bool le_pos(float x, float c) { return x <= c; }

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

// Speed c = sqrt(g h) of the boundary state of an imposed discharge
// (Sec. 2.2): the invariant w - 2c leaving the domain (R) and w = q / h
// give p(c) = 2c^3 + R c^2 - Q = 0 with Q = q g.  For Q > 0 the positive
// root is unique and p is increasing and convex to its right; Newton's
// iteration starts above it, at (max(-R, 0) + (Q/2)^{1/3}) (1 + 1/16), and
// decreases monotonically until an update no longer decreases c.
template <typename T>
__device__ __forceinline__ T inflow_celerity(T R, T Q)
{
    if (!(Q > T(0))) return R < T(0) ? T(-0.5) * R : T(0);
    T a = R < T(0) ? -R : T(0);
    T x = T(0.5) * Q;
    T y = icbrt(x);                       // x^{-1/3}
    T c = (a + x * y * y) * T(1.0625);
    for (int it = 0; it < 64; ++it) {
        T p = (T(2) * c + R) * (c * c) - Q;
        T dp = (T(6) * c + T(2) * R) * c;
        T cn = c - p / dp;
        if (!(cn < c)) break;
        c = cn;
    }
    return c;
}

// Boundary state of an imposed edge from its edge cell (Sec. 2.2): depth
// h1, normal discharge qn1 (positive into the domain), tangential discharge
// qt1 -> (hb, qnb, qtb).  The invariant R = w1 - 2 sqrt(g h1) leaving the
// domain is kept, the imposed value replaces the entering one; a torrential
// inflow (HQ) imposes both.  Out of line: only edge cells call it, and a
// call keeps its code out of the column sweep's register allocation.
template <typename T>
__device__ __noinline__ void imposed_state(const Params &P, int side, T h1, T qn1, T qt1, T &hb, T &qnb, T &qtb)
{
    const Scal<T> C = scal<T>(P);
    T bh, bq;
    if constexpr (std::is_same<T, double>::value) {
        bh = P.bc_h[side];
        bq = P.bc_q[side];
    } else {
        bh = P.fbc_h[side];
        bq = P.fbc_q[side];
    }
    T w1 = T(0), t1 = T(0);
    if (h1 > C.hdry) {
        T r = rcp(h1);
        w1 = qn1 * r;
        t1 = qt1 * r;
    }
    T R = w1 - T(2) * sq(C.g * h1);
    const int type = P.bc[side];
    if (type == SWOF_BC_IMPOSED_HQ) {
        hb = bh;
        qnb = bq;
        qtb = T(0);
    } else if (type == SWOF_BC_IMPOSED_H) {
        T w = R + T(2) * sq(C.g * bh);
        hb = bh;
        qnb = bh * w;
        qtb = bh * t1;
    } else {
        T c = inflow_celerity(R, bq * C.g);
        T h = (c * c) / C.g;
        hb = h;
        qnb = bq;
        qtb = h * t1;
    }
}

template <typename T>
struct Rec {
    T hm, hp, zm, zp, unm, unp, utm, utp;
};

// First order (Sec. 3.3): the face values are the cell values (z_- = z_+,
// so the centred term Fc vanishes).  FP32: z relative to the cell = 0.
template <typename T>
__device__ __forceinline__ Rec<T> rec1(T h, T z, T un, T ut)
{
    return {h, h, z, z, un, un, ut, ut};
}

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
    if (gt_pos(h1, hdry)) {
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
    if (gt_pos(h1, hdry)) {
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
    if (is0(hL) && is0(hR)) {
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

// Index checks of the debug build (SWOF_BOUNDS_CHECK): a failed check
// latches SWOF_EBOUNDS in the context's status word and the caller uses a
// safe value instead.  Compiled out otherwise.
__device__ __forceinline__ bool bounds_ok(const Params &P, bool ok)
{
    if constexpr (SWOF_BOUNDS_CHECK) {
        if (!ok && P.status) atomicCAS(P.status, 0, SWOF_EBOUNDS);
        return ok;
    } else {
        (void)P;
        return true;
    }
}

// Element of cell (gi, gj), gi in [-2, nx + 1 + padding], gj in [-2, ny + 1],
// of a padded field.
__device__ __forceinline__ size_t pidx(const Params &P, int gi, int gj)
{
    if constexpr (SWOF_BOUNDS_CHECK) {
        if (!bounds_ok(P, gj >= -2 && gj <= P.ny + 1 && gi + P.lpad >= 0 && gi + P.lpad < P.pitch)) return 0;
    }
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
            if (gt_pos(h, C.hdry)) {
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
                T ax, ay;
                if (P.order == 1) {           // cell values (Eq. (cfl), first order)
                    T cm = sq(C.g * m.x);
                    ax = ab(m.y) + cm;
                    ay = ab(m.z) + cm;
                } else {
                    ax = cell_speed(w.x, m.x, e.x, w.y, m.y, e.y, m.w, C.hdry, C.g);
                    ay = cell_speed(s_.x, m.x, n.x, s_.z, m.z, n.z, m.w, C.hdry, C.g);
                }
                kx = kmax(kx, speed_key(ax));
                ky = kmax(ky, speed_key(ay));
                // an imposed edge's boundary state (the ghost beside the edge cell)
                if (gi == 0 && P.bc[0] >= SWOF_BC_IMPOSED_H) kx = kmax(kx, speed_key(ab(w.y) + sq(C.g * w.x)));
                if (gi == P.nx - 1 && P.bc[1] >= SWOF_BC_IMPOSED_H) kx = kmax(kx, speed_key(ab(e.y) + sq(C.g * e.x)));
                if (gj == 0 && P.bc[2] >= SWOF_BC_IMPOSED_H) ky = kmax(ky, speed_key(ab(s_.z) + sq(C.g * s_.x)));
                if (gj == P.ny - 1 && P.bc[3] >= SWOF_BC_IMPOSED_H) ky = kmax(ky, speed_key(ab(n.z) + sq(C.g * n.x)));
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
    if (gt_pos(h, hdry)) {
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
    // Items: groups of rows for the x speeds on the ring columns (each thread
    // keeps one ring column), then (ring row, NT-column chunk) pairs for the
    // y speeds; blocks stride over both in one loop so the work is balanced.
    // One division per item, none per cell.
    const int nc = F.n_ring_cols;
    const int rows_per = nc > 0 ? (NT / nc > 0 ? NT / nc : 1) : 1;
    const int tr = nc > 0 ? threadIdx.x / nc : 0, c = nc > 0 ? threadIdx.x % nc : 0;
    const int items_x = nc > 0 ? (P.ny + rows_per - 1) / rows_per : 0;
    const int chunks = (P.nx + NT - 1) / NT;
    const int items = items_x + F.n_ring_rows * chunks;
    for (int it = blockIdx.x; it < items; it += gridDim.x) {
        if (it < items_x) {
            const int gj = it * rows_per + tr;
            if (tr >= rows_per || gj >= P.ny) continue;
            for (int cc = c; cc < nc; cc += NT) {
                const int gi = F.ring_cols[cc];
                V4<T> w = cell_rec(P, F, gi - 1, gj, C.hdry), m = cell_rec(P, F, gi, gj, C.hdry),
                      e = cell_rec(P, F, gi + 1, gj, C.hdry);
                if (!(is0(w.x) && is0(m.x) && is0(e.x)))   // three dry cells: speed 0
                    kx = kmax(kx, speed_key(cell_speed(w.x, m.x, e.x, w.y, m.y, e.y, m.w, C.hdry, C.g)));
                if (gi == 0 && P.bc[0] >= SWOF_BC_IMPOSED_H) kx = kmax(kx, speed_key(ab(w.y) + sq(C.g * w.x)));
                if (gi == P.nx - 1 && P.bc[1] >= SWOF_BC_IMPOSED_H)
                    kx = kmax(kx, speed_key(ab(e.y) + sq(C.g * e.x)));
            }
        } else {
            const int iy = it - items_x;
            const int q = iy / chunks, gi = (iy - q * chunks) * NT + threadIdx.x;
            if (gi >= P.nx) continue;
            const int gj = F.ring_rows[q];
            V4<T> s_ = cell_rec(P, F, gi, gj - 1, C.hdry), m = cell_rec(P, F, gi, gj, C.hdry),
                  n = cell_rec(P, F, gi, gj + 1, C.hdry);
            if (!(is0(s_.x) && is0(m.x) && is0(n.x)))
                ky = kmax(ky, speed_key(cell_speed(s_.x, m.x, n.x, s_.z, m.z, n.z, m.w, C.hdry, C.g)));
            if (gj == 0 && P.bc[2] >= SWOF_BC_IMPOSED_H) ky = kmax(ky, speed_key(ab(s_.z) + sq(C.g * s_.x)));
            if (gj == P.ny - 1 && P.bc[3] >= SWOF_BC_IMPOSED_H) ky = kmax(ky, speed_key(ab(n.z) + sq(C.g * n.x)));
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
// Ghost cells mirroring interior cell (gi, gj) of a state (Sec. 2.2): wall =
// mirror image with the normal discharge negated (two layers), outflow =
// edge cell extended, imposed = the boundary state of the edge cell in both
// layers.  x: the W/E edges, y: the S/N edges.  IMPOSED = false writes an
// imposed edge's ghosts as an outflow edge's (zero-filled tiles, which never
// touch an imposed edge).
template <typename T, bool IMPOSED = true>
__device__ __forceinline__ void ghosts_x(const Params &P, T *h, T *qx, T *qy, int gi, int gj, T hv, T qxv, T qyv)
{
    if (gi < 2) {            // west
        if (P.bc[0] == SWOF_BC_WALL) {
            size_t g = pidx(P, -1 - gi, gj);
            h[g] = hv; qx[g] = -qxv; qy[g] = qyv;
        } else if (gi == 0) {
            T gh = hv, gqx = qxv, gqy = qyv;
            if (IMPOSED && P.bc[0] >= SWOF_BC_IMPOSED_H) imposed_state<T>(P, 0, hv, qxv, qyv, gh, gqx, gqy);
            size_t g1 = pidx(P, -1, gj), g2 = pidx(P, -2, gj);
            h[g1] = gh; qx[g1] = gqx; qy[g1] = gqy;
            h[g2] = gh; qx[g2] = gqx; qy[g2] = gqy;
        }
    }
    if (gi >= P.nx - 2) {    // east
        if (P.bc[1] == SWOF_BC_WALL) {
            size_t g = pidx(P, 2 * P.nx - 1 - gi, gj);
            h[g] = hv; qx[g] = -qxv; qy[g] = qyv;
        } else if (gi == P.nx - 1) {
            T gh = hv, gqx = qxv, gqy = qyv;
            if (IMPOSED && P.bc[1] >= SWOF_BC_IMPOSED_H) {
                T qn;
                imposed_state<T>(P, 1, hv, -qxv, qyv, gh, qn, gqy);
                gqx = -qn;
            }
            size_t g1 = pidx(P, P.nx, gj), g2 = pidx(P, P.nx + 1, gj);
            h[g1] = gh; qx[g1] = gqx; qy[g1] = gqy;
            h[g2] = gh; qx[g2] = gqx; qy[g2] = gqy;
        }
    }
}
template <typename T, bool IMPOSED = true>
__device__ __forceinline__ void ghosts_y(const Params &P, T *h, T *qx, T *qy, int gi, int gj, T hv, T qxv, T qyv)
{
    if (gj < 2) {            // south
        if (P.bc[2] == SWOF_BC_WALL) {
            size_t g = pidx(P, gi, -1 - gj);
            h[g] = hv; qx[g] = qxv; qy[g] = -qyv;
        } else if (gj == 0) {
            T gh = hv, gqx = qxv, gqy = qyv;
            if (IMPOSED && P.bc[2] >= SWOF_BC_IMPOSED_H) imposed_state<T>(P, 2, hv, qyv, qxv, gh, gqy, gqx);
            size_t g1 = pidx(P, gi, -1), g2 = pidx(P, gi, -2);
            h[g1] = gh; qx[g1] = gqx; qy[g1] = gqy;
            h[g2] = gh; qx[g2] = gqx; qy[g2] = gqy;
        }
    }
    if (gj >= P.ny - 2) {    // north
        if (P.bc[3] == SWOF_BC_WALL) {
            size_t g = pidx(P, gi, 2 * P.ny - 1 - gj);
            h[g] = hv; qx[g] = qxv; qy[g] = -qyv;
        } else if (gj == P.ny - 1) {
            T gh = hv, gqx = qxv, gqy = qyv;
            if (IMPOSED && P.bc[3] >= SWOF_BC_IMPOSED_H) {
                T qn;
                imposed_state<T>(P, 3, hv, -qyv, qxv, gh, qn, gqx);
                gqy = -qn;
            }
            size_t g1 = pidx(P, gi, P.ny), g2 = pidx(P, gi, P.ny + 1);
            h[g1] = gh; qx[g1] = gqx; qy[g1] = gqy;
            h[g2] = gh; qx[g2] = gqx; qy[g2] = gqy;
        }
    }
}

// Write one interior cell of a stage output and the ghost cells it defines.
template <typename T, bool IMPOSED = true>
__device__ __forceinline__ void store_cell(const Params &P, T *h, T *qx, T *qy, int gi, int gj,
                                           T hv, T qxv, T qyv)
{
    size_t o = pidx(P, gi, gj);
    h[o] = hv;
    qx[o] = qxv;
    qy[o] = qyv;
    ghosts_x<T, IMPOSED>(P, h, qx, qy, gi, gj, hv, qxv, qyv);
    ghosts_y<T, IMPOSED>(P, h, qx, qy, gi, gj, hv, qxv, qyv);
}

// ---------------------------------------------------------------------------
// Ghost cells of U^n from its interior (after a state is set): thread k < ny
// does the W/E ghosts of row k, the next nx threads the S/N ghosts of one
// column each.
template <typename T>
__global__ void k_ghosts(Params P, Fields<T> F)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < P.ny) {
        const int gj = k;
        const int cols[4] = {0, 1, P.nx - 2, P.nx - 1};
        for (int c = 0; c < 4; ++c) {
            size_t o = pidx(P, cols[c], gj);
            ghosts_x(P, F.h, F.qx, F.qy, cols[c], gj, F.h[o], F.qx[o], F.qy[o]);
        }
    } else if (k < P.ny + P.nx) {
        const int gi = k - P.ny;
        const int rows[4] = {0, 1, P.ny - 2, P.ny - 1};
        for (int r = 0; r < 4; ++r) {
            size_t o = pidx(P, gi, rows[r]);
            ghosts_y(P, F.h, F.qx, F.qy, gi, rows[r], F.h[o], F.qx[o], F.qy[o]);
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

SWOF_KERNELS_END
#include "swof_sweep.cuh"
SWOF_KERNELS_BEGIN

// ---------------------------------------------------------------------------
// End of a first-order step (Sec. 3.3): U^{n+1} = U* of the single Euler
// stage, then rain, Green-Ampt and the dry clean-up in the order used after
// the Heun average, the ghosts, and the wave
// speeds of U^{n+1} on the cell values (plus an imposed edge's boundary
// state) for the next step's dt; with the CFL check on, the same speeds of
// U* first.  Blocks stride over rows, threads over the cells of a row.
template <typename T>
__device__ __forceinline__ void o1_speed(T h, T qx, T qy, T hdry, T g, T &ax, T &ay)
{
    T u = T(0), v = T(0);
    if (h > hdry) {
        T r = rcp(h);
        u = qx * r;
        v = qy * r;
    }
    T c = sq(g * h);
    ax = ab(u) + c;
    ay = ab(v) + c;
}

// max speed of the ghosts an imposed edge holds beside cell (gi, gj)
template <typename T, typename K>
__device__ __forceinline__ void o1_ghost_speeds(const Params &P, const T *h, const T *qx, const T *qy, int gi, int gj,
                                                T hdry, T g, K &kx, K &ky)
{
    T ax, ay;
    if (gi == 0 && P.bc[0] >= SWOF_BC_IMPOSED_H) {
        size_t o = pidx(P, -1, gj);
        o1_speed(h[o], qx[o], qy[o], hdry, g, ax, ay);
        kx = kmax(kx, speed_key(ax));
    }
    if (gi == P.nx - 1 && P.bc[1] >= SWOF_BC_IMPOSED_H) {
        size_t o = pidx(P, P.nx, gj);
        o1_speed(h[o], qx[o], qy[o], hdry, g, ax, ay);
        kx = kmax(kx, speed_key(ax));
    }
    if (gj == 0 && P.bc[2] >= SWOF_BC_IMPOSED_H) {
        size_t o = pidx(P, gi, -1);
        o1_speed(h[o], qx[o], qy[o], hdry, g, ax, ay);
        ky = kmax(ky, speed_key(ay));
    }
    if (gj == P.ny - 1 && P.bc[3] >= SWOF_BC_IMPOSED_H) {
        size_t o = pidx(P, gi, P.ny);
        o1_speed(h[o], qx[o], qy[o], hdry, g, ax, ay);
        ky = kmax(ky, speed_key(ay));
    }
}

template <typename T>
__global__ void __launch_bounds__(NT) k_commit1(Params P, Fields<T> F)
{
    using K = decltype(speed_key(T(0)));
    __shared__ K red[2][NW];
    __shared__ double sred[NW];
    DevCtl *ctl = F.ctl;
    if (ctl->status) return;
    const Scal<T> C = scal<T>(P);
    T dt, rdt;
    if constexpr (std::is_same<T, double>::value) {
        dt = ctl->dt; rdt = ctl->rdt;
    } else {
        dt = ctl->fdt; rdt = ctl->frdt;
    }
    const bool rain = ctl->rain_active != 0;
    K kx = 0, ky = 0, cx = 0, cy = 0;
    T infacc = T(0);
    for (int gj = blockIdx.x; gj < P.ny; gj += gridDim.x)
    for (int gi = threadIdx.x; gi < P.nx; gi += NT) {
        const size_t o = pidx(P, gi, gj);
        T h = F.h1[o], qx = F.qx1[o], qy = F.qy1[o];
        T ax, ay;
        if (P.check_cfl) {
            o1_speed(h, qx, qy, C.hdry, C.g, ax, ay);
            cx = kmax(cx, speed_key(ax));
            cy = kmax(cy, speed_key(ay));
            o1_ghost_speeds(P, F.h1, F.qx1, F.qy1, gi, gj, C.hdry, C.g, cx, cy);
        }
        if (rain) h = h + rdt;
        if (P.infiltration) {
            T vi = F.vinf[o];
            T ks = F.ksmap ? F.ksmap[o] : C.ks;
            T d;
            if (vi > T(0)) {
                T ic = ks * (T(1) + ((C.psi + h) * C.dtheta) / vi);
                d = mn(h, dt * ic);
            } else {
                d = h;
            }
            h = h - d;
            F.vinf[o] = vi + d;
            infacc += d;
        }
        if (h <= C.hdry) {
            qx = T(0);
            qy = T(0);
        }
        store_cell<T>(P, F.h, F.qx, F.qy, gi, gj, h, qx, qy);
        o1_speed(h, qx, qy, C.hdry, C.g, ax, ay);
        kx = kmax(kx, speed_key(ax));
        ky = kmax(ky, speed_key(ay));
        o1_ghost_speeds(P, F.h, F.qx, F.qy, gi, gj, C.hdry, C.g, kx, ky);
    }
    if (P.infiltration && !P.no_budget) {
        double s = block_sum_t(infacc, sred);
        if (threadIdx.x == 0) F.infil_slots[blockIdx.x] += s;
    }
    kx = block_max(kx, red[0]);
    ky = block_max(ky, red[1]);
    if (threadIdx.x == 0) {
        atomicMax(&ctl->lam_bits[0], key64(kx));
        atomicMax(&ctl->lam_bits[1], key64(ky));
    }
    if (P.check_cfl) {
        cx = block_max(cx, red[0]);
        cy = block_max(cy, red[1]);
        if (threadIdx.x == 0) {
            atomicMax(&ctl->lam2_bits[0], key64(cx));
            atomicMax(&ctl->lam2_bits[1], key64(cy));
            __threadfence();
            if (atomicAdd(&ctl->done2, 1u) == gridDim.x - 1) {
                __threadfence();
                double lx = __longlong_as_double((long long)atomicAdd(&ctl->lam2_bits[0], 0ull));
                double ly = __longlong_as_double((long long)atomicAdd(&ctl->lam2_bits[1], 0ull));
                ctl->lam2_bits[0] = 0ull;
                ctl->lam2_bits[1] = 0ull;
                ctl->done2 = 0u;
                if (ctl->dt * (lx / P.dx + ly / P.dy) > P.cfl) ctl->cfl_viol++;
            }
        }
    }
}

// Gauge record after a step: t, then (h, hu, hv) of each gauge cell (FP64).
template <typename T>
__global__ void k_gauges(Params P, Fields<T> F)
{
    DevCtl *ctl = F.ctl;
    if (ctl->status) return;
    const long long n = ctl->gauge_n;
    if (n >= F.gauge_cap) return;
    double *r = F.gauge_rec + n * (1 + 3LL * F.n_gauges);
    for (int g = threadIdx.x; g < F.n_gauges; g += blockDim.x) {
        const long long o = F.gauge_off[g];
        r[1 + 3 * g] = (double)F.h[o];
        r[2 + 3 * g] = (double)F.qx[o];
        r[3 + 3 * g] = (double)F.qy[o];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        r[0] = ctl->t;
        ctl->gauge_n = n + 1;
    }
}

// Running maximum depth after a step (only while it is tracked): one pass
// over the interior, hmax = max(hmax, h).
template <typename T>
__global__ void k_hmax(Params P, const T *h, T *hmax)
{
    for (int gj = blockIdx.x; gj < P.ny; gj += gridDim.x)
        for (int gi = threadIdx.x; gi < P.nx; gi += blockDim.x) {
            size_t o = pidx(P, gi, gj);
            hmax[o] = mx(hmax[o], h[o]);
        }
}

// Interior of one padded field -> dense [ny][nx] FP64.
template <typename T>
__global__ void k_pack1(Params P, const T *src, double *dst)
{
    size_t n = (size_t)P.nx * P.ny;
    for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x)
        dst[k] = (double)src[pidx(P, (int)(k % P.nx), (int)(k / P.nx))];
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
int launch_lambda_ring_t(const Params &P, void *f, void *stream)
{
    const Fields<T> &F = *static_cast<const Fields<T> *>(f);
    long long total = (long long)F.n_ring_cols * P.ny + (long long)F.n_ring_rows * P.nx;
    long long b = (total + NT - 1) / NT;
    int grid = (int)(b < 152 * 8 ? (b > 0 ? b : 1) : 152 * 8);
    k_lambda_ring<T><<<grid, NT, 0, (cudaStream_t)stream>>>(P, F);
    return (int)cudaGetLastError();
}

// Per-device attributes: every stage kernel's input ring sits in dynamic
// shared memory beyond the default 48 KB window, so each instantiation is
// opted in on the current device.
template <typename T, int STAGE, int NTX, int H, bool ORD1 = false>
cudaError_t sweep_opt_in()
{
    return cudaFuncSetAttribute(k_sweep<T, STAGE, NTX, H, ORD1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)ring_bytes<T, STAGE, NTX>());
}

template <typename T, int NTX, int H>
cudaError_t sweep_opt_in_shape()
{
    cudaError_t e = sweep_opt_in<T, 1, NTX, H>();
    if (e == cudaSuccess) e = sweep_opt_in<T, 2, NTX, H>();
    if (e == cudaSuccess) e = sweep_opt_in<T, 1, NTX, H, true>();
    return e;
}

template <typename T>
int configure_t()
{
    cudaError_t e = sweep_opt_in_shape<T, 128, 32>();
    if (e == cudaSuccess) e = sweep_opt_in_shape<T, 128, 64>();
    if (e == cudaSuccess) e = sweep_opt_in_shape<T, 256, 32>();
    if (e == cudaSuccess) e = sweep_opt_in_shape<T, 64, 64>();
    if (e == cudaSuccess) e = sweep_opt_in_shape<T, 64, 16>();
    return (int)e;
}

template <typename T, int STAGE, int NTX, int H>
int launch_sweep(const Params &P, const Fields<T> &F, cudaStream_t s)
{
    dim3 grid((P.nx + NTX - 5) / (NTX - 4), (P.ny + H - 1) / H);
    k_sweep<T, STAGE, NTX, H><<<grid, NTX, ring_bytes<T, STAGE, NTX>(), s>>>(P, F, F.tmaps[map_width_index(NTX)]);
    return (int)cudaGetLastError();
}

// The register-prefetch forms (shapes N_RING_SHAPES..), compiled in their
// own translation units (swof_fp32_reg.cu, swof_fp64_reg.cu).
template <typename T, int STAGE, int NTX, int H, bool ORD1>
int launch_sweep_reg(const Params &P, const Fields<T> &F, cudaStream_t s)
{
    dim3 grid((P.nx + NTX - 5) / (NTX - 4), (P.ny + H - 1) / H);
    k_sweep_reg<T, STAGE, NTX, H, ORD1><<<grid, NTX, 0, s>>>(P, F);
    return (int)cudaGetLastError();
}
template <typename T, int STAGE, bool ORD1>
int launch_stage_reg(int cfg, const Params &P, const Fields<T> &F, cudaStream_t s);

template <typename T, int STAGE>
int launch_stage_t(const Params &P, void *f, void *stream)
{
    const Fields<T> &F = *static_cast<const Fields<T> *>(f);
    cudaStream_t s = (cudaStream_t)stream;
    const int cfg = STAGE == 1 ? P.tile_cfg : P.tile_cfg2;
    if (cfg >= N_RING_SHAPES) return launch_stage_reg<T, STAGE, false>(cfg, P, F, s);
    switch (cfg) {
    case 1: return launch_sweep<T, STAGE, 128, 64>(P, F, s);
    case 2: return launch_sweep<T, STAGE, 256, 32>(P, F, s);
    case 3: return launch_sweep<T, STAGE, 64, 64>(P, F, s);
    case 4: return launch_sweep<T, STAGE, 64, 16>(P, F, s);
    default: return launch_sweep<T, STAGE, 128, 32>(P, F, s);
    }
}

template <typename T, int NTX, int H>
int launch_sweep_o1(const Params &P, const Fields<T> &F, cudaStream_t s)
{
    dim3 grid((P.nx + NTX - 5) / (NTX - 4), (P.ny + H - 1) / H);
    k_sweep<T, 1, NTX, H, true><<<grid, NTX, ring_bytes<T, 1, NTX>(), s>>>(P, F, F.tmaps[map_width_index(NTX)]);
    return (int)cudaGetLastError();
}

template <typename T>
int launch_stage1_o1_t(const Params &P, void *f, void *stream)
{
    const Fields<T> &F = *static_cast<const Fields<T> *>(f);
    cudaStream_t s = (cudaStream_t)stream;
    if (P.tile_cfg >= N_RING_SHAPES) return launch_stage_reg<T, 1, true>(P.tile_cfg, P, F, s);
    switch (P.tile_cfg) {
    case 1: return launch_sweep_o1<T, 128, 64>(P, F, s);
    case 2: return launch_sweep_o1<T, 256, 32>(P, F, s);
    case 3: return launch_sweep_o1<T, 64, 64>(P, F, s);
    case 4: return launch_sweep_o1<T, 64, 16>(P, F, s);
    default: return launch_sweep_o1<T, 128, 32>(P, F, s);
    }
}

// grid of the first-order commit: at most one block per budget slot
template <typename T>
int launch_commit_o1_t(const Params &P, void *f, void *stream)
{
    const Fields<T> &F = *static_cast<const Fields<T> *>(f);
    // one block per row (up to the number of budget slots): enough loads in
    // flight to stream the 24 B per cell (FP32) of the step end
    long long b = P.ny;
    long long slots = max_stage_blocks(P.nx, P.ny);
    if (b > slots) b = slots;
    k_commit1<T><<<(int)b, NT, 0, (cudaStream_t)stream>>>(P, F);
    return (int)cudaGetLastError();
}

template <typename T>
int launch_gauges_t(const Params &P, void *f, void *stream)
{
    const Fields<T> &F = *static_cast<const Fields<T> *>(f);
    k_gauges<T><<<1, 256, 0, (cudaStream_t)stream>>>(P, F);
    return (int)cudaGetLastError();
}

template <typename T>
int launch_hmax_t(const Params &P, void *f, void *stream)
{
    const Fields<T> &F = *static_cast<const Fields<T> *>(f);
    int b = P.ny < 152 * 8 ? P.ny : 152 * 8;
    k_hmax<T><<<b, 256, 0, (cudaStream_t)stream>>>(P, F.h, F.hmax);
    return (int)cudaGetLastError();
}

template <typename T>
int launch_pack1_t(const Params &P, const void *src, double *dst, void *stream)
{
    k_pack1<T><<<1216, 256, 0, (cudaStream_t)stream>>>(P, (const T *)src, dst);
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

inline int stage_slots(const Params &P) { return max_stage_blocks(P.nx, P.ny); }

// One thread forms the padded index of cell (i, j) through pidx() and reads
// the depth there (debug build: a failed check reads element 0 instead).
template <typename T>
__global__ void k_probe(Params P, Fields<T> F, int i, int j)
{
    const size_t o = pidx(P, i, j);
    volatile T x = F.h[o];
    (void)x;
}

template <typename T>
int launch_probe_t(const Params &P, void *f, int i, int j, void *stream)
{
    const Fields<T> &F = *static_cast<const Fields<T> *>(f);
    k_probe<T><<<1, 1, 0, (cudaStream_t)stream>>>(P, F, i, j);
    return (int)cudaGetLastError();
}

SWOF_KERNELS_END

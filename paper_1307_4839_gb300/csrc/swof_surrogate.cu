// swof_surrogate.cu -- the learned surrogate's serving path around the
// network of swof_unet.cu: coarsening of a solver state (the surrogate's
// training data and its judge), per-member budget statistics, and the
// rollout driver that advances a batch of coarse members one time span per
// network call, checks each prediction for positivity and mass balance, and
// falls back to the plain solver (the scheme of Sec. 2-3 on the coarse
// grid) for every member whose check fails.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "swof_ctx.h"

// network dimensions {in_ch, out_ch, H, W, max_batch} (swof_unet.cu)
void swof_unet_dims(const swof_unet *u, int *d);

namespace {

using namespace swof;

int cuerr(cudaError_t e) { return e == cudaSuccess ? SWOF_OK : SWOF_ECUDA; }

int grid_for(long long n)
{
    long long g = (n + 255) / 256;
    return (int)(g < 152 * 16 ? (g > 0 ? g : 1) : 152 * 16);
}

// Block means over f x f cells of h, qx, qy and the infiltrated depth into
// out [4][ny/f][nx/f] (fp32).  The sum runs in FP64 in a fixed order.
template <typename T>
__global__ void k_coarsen(Params P, Fields<T> F, int f, float *out)
{
    const int cx = P.nx / f, cy = P.ny / f;
    const long long plane = (long long)cx * cy, total = 4 * plane;
    const double inv = 1.0 / ((double)f * f);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int ch = (int)(i / plane);
        const long long r = i - ch * plane;
        const int J = (int)(r / cx), I = (int)(r - (long long)J * cx);
        const T *a = ch == 0 ? F.h : ch == 1 ? F.qx : ch == 2 ? F.qy : F.vinf;
        double s = 0.0;
        for (int dj = 0; dj < f; ++dj)
            for (int di = 0; di < f; ++di)
                s += (double)a[(size_t)(J * f + dj + 2) * P.pitch + (size_t)(I * f + di + P.lpad)];
        out[i] = (float)(s * inv);
    }
}

// Block mean over the f x f fine cells of coarse cell (I, J) of a dense
// [ny][nx] field (FP64 sum in a fixed order).
__device__ __forceinline__ double block_mean(const double *a, int nx, int f, int I, int J)
{
    double s = 0.0;
    for (int dj = 0; dj < f; ++dj)
        for (int di = 0; di < f; ++di) s += a[(size_t)(J * f + dj) * nx + (size_t)(I * f + di)];
    return s / ((double)f * f);
}

// The surrogate's static channels per coarse cell: the slopes of the
// block-mean bed (central differences, one-sided at the edges, spacing
// f dx and f dy -- each thread recomputes its neighbours' block means) and
// the block-mean K_s, written to every snapshot.
__global__ void k_coarsen_static(const double *z, const double *ks, double ks_const, int nx, int ny, double dx,
                                 double dy, int f, float *out, long long snap_stride, int nsnap)
{
    const int cx = nx / f, cy = ny / f;
    const long long plane = (long long)cx * cy;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < plane;
         i += (long long)gridDim.x * blockDim.x) {
        const int J = (int)(i / cx), I = (int)(i - (long long)J * cx);
        const int Iw = I > 0 ? I - 1 : I, Ie = I < cx - 1 ? I + 1 : I;
        const int Js = J > 0 ? J - 1 : J, Jn = J < cy - 1 ? J + 1 : J;
        const double zx = (block_mean(z, nx, f, Ie, J) - block_mean(z, nx, f, Iw, J)) / ((double)(Ie - Iw) * f * dx);
        const double zy = (block_mean(z, nx, f, I, Jn) - block_mean(z, nx, f, I, Js)) / ((double)(Jn - Js) * f * dy);
        const double kc = ks ? block_mean(ks, nx, f, I, J) : ks_const;
        for (int k = 0; k < nsnap; ++k) {
            float *o = out + (long long)k * snap_stride;
            o[i] = (float)zx;
            o[plane + i] = (float)zy;
            o[2 * plane + i] = (float)kc;
        }
    }
}

// One block per member b of states [B][C][H][W] (channels h, hu, hv, then
// V_inf when C >= 4).  out[5b .. 5b+4] = {sum h, sum min(h, 0), discharge
// out of the domain through the edges flagged in outmask [m^3/s], sum V_inf,
// min h}.  outmask bits: 1 W (i = 0), 2 E (i = W-1), 4 S (j = 0), 8 N
// (j = H-1); the discharge is sum q_normal * edge length.  FP64 sums in a
// fixed order (thread strides, then a fixed tree).
__global__ void k_batch_stats(const float *st, int C, int H, int W, int outmask, double dx, double dy,
                              double *out)
{
    __shared__ double red[5][8];
    const int b = blockIdx.x;
    const long long HW = (long long)H * W;
    const float *h = st + (size_t)b * C * HW, *qx = h + HW, *qy = h + 2 * HW;
    const float *vi = C >= 4 ? h + 3 * HW : nullptr;
    double s = 0.0, neg = 0.0, q = 0.0, sv = 0.0, mn = INFINITY;
    for (long long i = threadIdx.x; i < HW; i += blockDim.x) {
        const double v = h[i];
        s += v;
        neg += fmin(v, 0.0);
        mn = fmin(mn, v);
        if (vi) sv += (double)vi[i];
    }
    for (int i = threadIdx.x; i < W; i += blockDim.x) {
        if (outmask & 8) q += (double)qy[(size_t)(H - 1) * W + i] * dx;
        if (outmask & 4) q -= (double)qy[i] * dx;
    }
    for (int j = threadIdx.x; j < H; j += blockDim.x) {
        if (outmask & 2) q += (double)qx[(size_t)j * W + W - 1] * dy;
        if (outmask & 1) q -= (double)qx[(size_t)j * W] * dy;
    }
    double v[5] = {s, neg, q, sv, mn};
    for (int k = 0; k < 5; ++k)
        for (int o = 16; o > 0; o >>= 1) {
            const double w = __shfl_xor_sync(0xffffffffu, v[k], o);
            v[k] = k == 4 ? fmin(v[k], w) : v[k] + w;
        }
    const int warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if ((threadIdx.x & 31) == 0)
        for (int k = 0; k < 5; ++k) red[k][warp] = v[k];
    __syncthreads();
    if (threadIdx.x < 5) {
        const int k = threadIdx.x;
        double a = red[k][0];
        for (int w = 1; w < nw; ++w) a = k == 4 ? fmin(a, red[k][w]) : a + red[k][w];
        out[5 * b + k] = a;
    }
}

// Accepted members take the prediction (h >= 0, q = 0 where h <= h_dry,
// V_inf never decreasing); every member gets the rain rate of its next span
// in channel rain_ch (< 0: none).
__global__ void k_commit(float *st, int C, const float *pred, int Co, long long HW, int B, const int *accept,
                         const float *rain, int rain_ch, float h_dry)
{
    const long long total = (long long)B * HW;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(i / HW);
        const long long p = i - (long long)b * HW;
        float *s = st + (size_t)b * C * HW + p;
        if (accept[b]) {
            const float *o = pred + (size_t)b * Co * HW + p;
            const float hn = fmaxf(o[0], 0.0f);
            const bool dry = hn <= h_dry;
            s[0] = hn;
            s[HW] = dry ? 0.0f : o[HW];
            s[2 * HW] = dry ? 0.0f : o[2 * HW];
            if (Co >= 4 && C >= 4) s[3 * HW] = fmaxf(o[3 * HW], s[3 * HW]);
        }
        if (rain_ch >= 0) s[(size_t)rain_ch * HW] = rain[b];
    }
}

// V_inf interior <-> dense [ny][nx] array of type S
template <typename T, typename S, bool TO_FIELD>
__global__ void k_vinf_copy(Params P, T *vinf, S *d)
{
    const long long n = (long long)P.nx * P.ny;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(i / P.nx), x = (int)(i - (long long)j * P.nx);
        T &f = vinf[(size_t)(j + 2) * P.pitch + (size_t)(x + P.lpad)];
        if (TO_FIELD)
            f = (T)d[i];
        else
            d[i] = (S)f;
    }
}

template <bool TO_FIELD>
int vinf_copy(swof_ctx *c, void *d, int dtype)
{
    const int g = grid_for((long long)c->P.nx * c->P.ny);
    if (c->prec == SWOF_FP64) {
        if (dtype == SWOF_FP64)
            k_vinf_copy<double, double, TO_FIELD><<<g, 256, 0, c->stream>>>(c->P, c->f64.vinf, (double *)d);
        else
            k_vinf_copy<double, float, TO_FIELD><<<g, 256, 0, c->stream>>>(c->P, c->f64.vinf, (float *)d);
    } else {
        if (dtype == SWOF_FP64)
            k_vinf_copy<float, double, TO_FIELD><<<g, 256, 0, c->stream>>>(c->P, c->f32.vinf, (double *)d);
        else
            k_vinf_copy<float, float, TO_FIELD><<<g, 256, 0, c->stream>>>(c->P, c->f32.vinf, (float *)d);
    }
    return cuerr(cudaGetLastError());
}

__global__ void k_add(float *a, long long n, float v)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        a[i] += v;
}

// Rain rate r[0] averaged over the n steps of length span / n from t0: the
// solver adds rain in a step when the step starts in [r[1], r[2]).
double span_rain(const double *r, double t0, double span, int n)
{
    int c = 0;
    for (int j = 0; j < n; ++j) {
        const double tj = t0 + j * (span / n);
        c += tj >= r[1] && tj < r[2];
    }
    return r[0] * c / n;
}

// Events owned by one rollout call: one on the rollout stream, one per
// fallback context used.
struct Events {
    cudaEvent_t main = nullptr;
    std::vector<std::pair<swof_ctx *, cudaEvent_t>> ctx;
    ~Events()
    {
        if (main) cudaEventDestroy(main);
        for (auto &p : ctx) cudaEventDestroy(p.second);
    }
    cudaEvent_t of(swof_ctx *c)
    {
        for (auto &p : ctx)
            if (p.first == c) return p.second;
        cudaEvent_t e = nullptr;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return nullptr;
        ctx.emplace_back(c, e);
        return e;
    }
};

struct Scratch {
    std::vector<void *> p;
    ~Scratch()
    {
        for (void *q : p) cudaFree(q);
    }
    template <typename T>
    T *get(size_t n)
    {
        void *q = nullptr;
        if (cudaMalloc(&q, n * sizeof(T) > 0 ? n * sizeof(T) : 1) != cudaSuccess) return nullptr;
        p.push_back(q);
        return static_cast<T *>(q);
    }
};

// A member slot (dense fp32 planes h, hu, hv[, V_inf] of H x W) into a
// context's padded state, with its time; the latched status and the wave-
// speed words are cleared (what swof_set_state_device + set_infiltrated +
// swof_set_time do, in one launch).
template <typename T>
__global__ void k_member_in(Params P, Fields<T> F, DevCtl *ctl, const float *sb, long long HW, int vinf, double t)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < HW; i += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(i / P.nx), x = (int)(i - (long long)j * P.nx);
        const size_t o = (size_t)(j + 2) * P.pitch + (size_t)(x + P.lpad);
        F.h[o] = (T)sb[i];
        F.qx[o] = (T)sb[HW + i];
        F.qy[o] = (T)sb[2 * HW + i];
        if (vinf) F.vinf[o] = (T)sb[3 * HW + i];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->t = t;
        ctl->status = 0;
        ctl->lam_bits[0] = 0ull;
        ctl->lam_bits[1] = 0ull;
    }
}

// The context's state (and V_inf) back into the member slot.
template <typename T>
__global__ void k_member_out(Params P, Fields<T> F, float *sb, long long HW, int vinf)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < HW; i += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(i / P.nx), x = (int)(i - (long long)j * P.nx);
        const size_t o = (size_t)(j + 2) * P.pitch + (size_t)(x + P.lpad);
        sb[i] = (float)F.h[o];
        sb[HW + i] = (float)F.qx[o];
        sb[2 * HW + i] = (float)F.qy[o];
        if (vinf) sb[3 * HW + i] = (float)F.vinf[o];
    }
}

// Enqueue, on the fallback context's stream, the plain solver's advance of
// member slot sb over the span: the context takes the member's pre-call
// state, V_inf and time, takes `steps` steps and writes its state back
// (four launches: load, ghosts, the n-step sequence, store).
int enqueue_fallback(swof_ctx *c, float *sb, int C, long long HW, int out_ch, double t, int steps)
{
    const int vinf = out_ch >= 4 && C >= 4;
    const int g = grid_for(HW);
    if (c->prec == SWOF_FP64)
        k_member_in<double><<<g, 256, 0, c->stream>>>(c->P, c->f64, c->ctl, sb, HW, vinf, t);
    else
        k_member_in<float><<<g, 256, 0, c->stream>>>(c->P, c->f32, c->ctl, sb, HW, vinf, t);
    int st = cuerr(cudaGetLastError());
    if (!st) st = cuerr((cudaError_t)c->L->ghosts(c->P, c->fields(), c->stream));
    c->lam_valid = false;
    if (!st) st = swof_step(c, steps, nullptr);
    if (st) return st;
    if (c->prec == SWOF_FP64)
        k_member_out<double><<<g, 256, 0, c->stream>>>(c->P, c->f64, sb, HW, vinf);
    else
        k_member_out<float><<<g, 256, 0, c->stream>>>(c->P, c->f32, sb, HW, vinf);
    return cuerr(cudaGetLastError());
}

}  // namespace

extern "C" {

int swof_coarsen(swof_ctx *c, int f, float *out)
{
    if (!c || !out || f < 1 || c->P.nx % f || c->P.ny % f) return SWOF_EINVAL;
    const long long n = 4LL * (c->P.nx / f) * (c->P.ny / f);
    if (c->prec == SWOF_FP64)
        k_coarsen<double><<<grid_for(n), 256, 0, c->stream>>>(c->P, c->f64, f, out);
    else
        k_coarsen<float><<<grid_for(n), 256, 0, c->stream>>>(c->P, c->f32, f, out);
    return cuerr(cudaGetLastError());
}

int swof_coarsen_static(const double *z, const double *ks, double ks_const, int nx, int ny, double dx, double dy,
                        int f, float *out, long long snap_stride, int nsnap, void *stream)
{
    if (!z || !out || f < 1 || nx % f || ny % f || nx / f < 2 || ny / f < 2 || !(dx > 0) || !(dy > 0) || nsnap < 1 ||
        snap_stride < 3LL * (nx / f) * (ny / f))
        return SWOF_EINVAL;
    const long long n = (long long)(nx / f) * (ny / f);
    k_coarsen_static<<<grid_for(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(z, ks, ks_const, nx, ny, dx, dy, f,
                                                                               out, snap_stride, nsnap);
    return cuerr(cudaGetLastError());
}

int swof_set_infiltrated_device(swof_ctx *c, const void *v, int dtype)
{
    if (!c || !v || (dtype != SWOF_FP64 && dtype != SWOF_FP32)) return SWOF_EINVAL;
    return vinf_copy<true>(c, const_cast<void *>(v), dtype);
}

int swof_get_infiltrated_device(swof_ctx *c, void *v, int dtype)
{
    if (!c || !v || (dtype != SWOF_FP64 && dtype != SWOF_FP32)) return SWOF_EINVAL;
    return vinf_copy<false>(c, v, dtype);
}

int swof_batch_stats(const float *states, int B, int C, int H, int W, int outmask, double dx, double dy,
                     double *out, void *stream)
{
    if (!states || !out || B < 1 || C < 3 || H < 1 || W < 1 || outmask < 0 || outmask > 15) return SWOF_EINVAL;
    k_batch_stats<<<B, 256, 0, static_cast<cudaStream_t>(stream)>>>(states, C, H, W, outmask, dx, dy, out);
    return cuerr(cudaGetLastError());
}

int swof_surrogate_rollout(swof_unet *u, float *states, int B, double *t, const double *rain,
                           swof_ctx *const *fallback, const int *fallback_of, const swof_rollout_opts *o,
                           int *accepted, double *checks, void *stream)
{
    if (!u || !states || B < 1 || !t || !rain || !o) return SWOF_EINVAL;
    int d[5];
    swof_unet_dims(u, d);
    const int C = d[0], Co = d[1], H = d[2], W = d[3], maxB = d[4];
    if (Co < 3 || Co > 4 || C < Co || o->calls < 0 || !(o->span > 0.0) || !(o->dx > 0.0) || !(o->dy > 0.0) ||
        !(o->tol > 0.0) || o->fallback_steps < 1 || o->rain_channel >= C || o->outflow_mask < 0 ||
        o->outflow_mask > 15 || (o->rain_channel >= 0 && o->rain_channel < Co))
        return SWOF_EINVAL;
    const long long HW = (long long)H * W;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Scratch m;
    float *pred = m.get<float>((size_t)B * Co * HW);
    double *stats = m.get<double>((size_t)10 * B);
    int *acc_d = m.get<int>(B);
    float *rain_d = m.get<float>(B);
    if (!pred || !stats || !acc_d || !rain_d) return SWOF_ENOMEM;
    std::vector<double> sh((size_t)10 * B);
    std::vector<float> rain_next(B);
    std::vector<int> acc(B);
    std::vector<swof_ctx *> used;
    const double A = o->dx * o->dy, area = A * (double)HW;
    int status = SWOF_OK;
    Events evs;
    if (cudaEventCreateWithFlags(&evs.main, cudaEventDisableTiming) != cudaSuccess) return SWOF_ECUDA;
    cudaEvent_t ev = evs.main;
    for (int k = 0; k < o->calls && status == SWOF_OK; ++k) {
        int st = swof_batch_stats(states, B, C, H, W, o->outflow_mask, o->dx, o->dy, stats, s);
        for (int b0 = 0; b0 < B && !st; b0 += maxB) {
            const int nb = B - b0 < maxB ? B - b0 : maxB;
            st = swof_surrogate_predict(u, states + (size_t)b0 * C * HW, nb, pred + (size_t)b0 * Co * HW, s);
        }
        if (st) return st;
        if (k == o->inject_call && o->inject_member >= 0 && o->inject_member < B)
            k_add<<<grid_for(HW), 256, 0, s>>>(pred + (size_t)o->inject_member * Co * HW, HW, (float)o->inject_dh);
        if ((st = swof_batch_stats(pred, B, Co, H, W, o->outflow_mask, o->dx, o->dy, stats + 5 * B, s))) return st;
        if (cudaMemcpyAsync(sh.data(), stats, sh.size() * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return SWOF_ECUDA;
        // Positivity and mass checks: the water volume change must equal
        // rain in - infiltration - discharge out (trapezoidal in time),
        // relative to the water present plus the rain of the span.
        for (int b = 0; b < B; ++b) {
            const double *pb = &sh[5 * b], *pa = &sh[5 * (B + b)];
            const double *rb = rain + 3 * b;
            const double R = span_rain(rb, t[b], o->span, o->fallback_steps) * o->span * area;
            const double I = Co >= 4 ? (pa[3] - pb[3]) * A : 0.0;
            const double Q = 0.5 * (pb[2] + pa[2]) * o->span;
            const double ref = fmax(pb[0] * A + R, area * o->h_dry);
            const double merr = fabs(pa[0] * A - pb[0] * A - (R - I - Q)) / ref;
            const double nerr = -pa[1] * A / ref;
            acc[b] = std::isfinite(merr) && std::isfinite(nerr) && merr <= o->tol && nerr <= o->tol;
            rain_next[b] = (float)span_rain(rb, t[b] + o->span, o->span, o->fallback_steps);
            if (checks) {
                checks[2 * ((size_t)k * B + b)] = merr;
                checks[2 * ((size_t)k * B + b) + 1] = nerr;
            }
            if (accepted) accepted[(size_t)k * B + b] = acc[b];
        }
        if (cudaMemcpyAsync(acc_d, acc.data(), B * sizeof(int), cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(rain_d, rain_next.data(), B * sizeof(float), cudaMemcpyHostToDevice, s) != cudaSuccess)
            return SWOF_ECUDA;
        k_commit<<<grid_for((long long)B * HW), 256, 0, s>>>(states, C, pred, Co, HW, B, acc_d, rain_d,
                                                              o->rain_channel, (float)o->h_dry);
        if (cudaEventRecord(ev, s) != cudaSuccess) return SWOF_ECUDA;
        // failing members: the plain solver on each fallback context's own
        // stream (after the commit), the rollout stream waiting for all
        used.clear();
        for (int b = 0; b < B; ++b) {
            if (!acc[b]) {
                const int fi = fallback && fallback_of ? fallback_of[b] : -1;
                swof_ctx *fc = fi >= 0 ? fallback[fi] : nullptr;
                if (!fc || fc->P.nx != W || fc->P.ny != H) {
                    status = SWOF_ESTATE;   // no solver to fall back on: this member stops here
                    continue;
                }
                if (std::find(used.begin(), used.end(), fc) == used.end()) {
                    if (cudaStreamWaitEvent(fc->stream, ev, 0) != cudaSuccess) return SWOF_ECUDA;
                    used.push_back(fc);
                }
                if ((st = enqueue_fallback(fc, states + (size_t)b * C * HW, C, HW, Co, t[b], o->fallback_steps)))
                    return st;
            }
            t[b] += o->span;
        }
        for (swof_ctx *fc : used) {
            cudaEvent_t e = evs.of(fc);
            if (!e || cudaEventRecord(e, fc->stream) != cudaSuccess || cudaStreamWaitEvent(s, e, 0) != cudaSuccess)
                return SWOF_ECUDA;
        }
    }
    // latched errors of the fallback solvers used (synchronises them)
    for (auto &p : evs.ctx) {
        swof_step_info info;
        int st = swof_step(p.first, 0, &info);
        if (st) return st;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return SWOF_ECUDA;
    return status;
}

}  // extern "C"

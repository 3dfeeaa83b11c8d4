// swof_api.cu -- host side of libswof: contexts, device memory, the C ABI
// declared in include/swof.h.  Arithmetic of the scheme lives in the
// kernels (swof_kernels.cuh); this file only lays out memory, converts
// host arrays and enqueues launches.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "swof_ctx.h"

namespace {

int cuda_err(cudaError_t e) { return e == cudaSuccess ? SWOF_OK : SWOF_ECUDA; }

template <typename T>
T *dalloc(swof_ctx *c, size_t n, int *st)
{
    void *p = nullptr;
    if (*st) return nullptr;
    if (cudaMalloc(&p, n * sizeof(T) > 0 ? n * sizeof(T) : 16) != cudaSuccess) {
        *st = SWOF_ENOMEM;
        return nullptr;
    }
    c->allocs.push_back(p);
    if (cudaMemsetAsync(p, 0, n * sizeof(T), c->stream) != cudaSuccess) *st = SWOF_ECUDA;
    return static_cast<T *>(p);
}

size_t padded_elems(const swof_ctx *c) { return (size_t)(c->P.ny + 4) * (size_t)c->P.pitch; }

// Host padded copy (double) of an interior [ny][nx] array, ghosts by the
// boundary rule (scalar fields: mirror at walls, extension at outflow).
std::vector<double> host_padded(const swof_ctx *c, const double *a)
{
    const Params &P = c->P;
    std::vector<double> out(padded_elems(c), 0.0);
    auto at = [&](int i, int j) -> double & {
        return out[(size_t)(j + 2) * P.pitch + (size_t)(i + P.lpad)];
    };
    for (int j = 0; j < P.ny; ++j)
        for (int i = 0; i < P.nx; ++i) at(i, j) = a[(size_t)j * P.nx + i];
    for (int j = 0; j < P.ny; ++j)
        for (int k = 0; k < 2; ++k) {
            at(-1 - k, j) = (P.bc[0] == SWOF_BC_WALL) ? at(k, j) : at(0, j);
            at(P.nx + k, j) = (P.bc[1] == SWOF_BC_WALL) ? at(P.nx - 1 - k, j) : at(P.nx - 1, j);
        }
    for (int i = 0; i < P.nx; ++i)
        for (int k = 0; k < 2; ++k) {
            at(i, -1 - k) = (P.bc[2] == SWOF_BC_WALL) ? at(i, k) : at(i, 0);
            at(i, P.ny + k) = (P.bc[3] == SWOF_BC_WALL) ? at(i, P.ny - 1 - k) : at(i, P.ny - 1);
        }
    return out;
}

template <typename T>
int upload_padded(swof_ctx *c, T *dst, const std::vector<double> &src)
{
    std::vector<T> tmp(src.size());
    for (size_t k = 0; k < src.size(); ++k) tmp[k] = (T)src[k];
    cudaError_t e = cudaMemcpyAsync(dst, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return cuda_err(e);
}

// Interior [ny][nx] host doubles -> padded device array of T (no ghosts).
template <typename T>
int upload_interior(swof_ctx *c, T *dst, const double *src)
{
    const Params &P = c->P;
    std::vector<T> tmp((size_t)P.nx * P.ny);
    for (size_t k = 0; k < tmp.size(); ++k) tmp[k] = (T)src[k];
    cudaError_t e = cudaMemcpy2DAsync(dst + 2 * (size_t)P.pitch + P.lpad, (size_t)P.pitch * sizeof(T),
                                      tmp.data(), (size_t)P.nx * sizeof(T), (size_t)P.nx * sizeof(T),
                                      (size_t)P.ny, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return cuda_err(e);
}

template <typename T>
int download_interior(swof_ctx *c, const T *src, double *dst)
{
    const Params &P = c->P;
    std::vector<T> tmp((size_t)P.nx * P.ny);
    cudaError_t e = cudaMemcpy2DAsync(tmp.data(), (size_t)P.nx * sizeof(T),
                                      src + 2 * (size_t)P.pitch + P.lpad, (size_t)P.pitch * sizeof(T),
                                      (size_t)P.nx * sizeof(T), (size_t)P.ny, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return SWOF_ECUDA;
    for (size_t k = 0; k < tmp.size(); ++k) dst[k] = (double)tmp[k];
    return SWOF_OK;
}

int read_ctl(swof_ctx *c, DevCtl *h)
{
    cudaError_t e = cudaMemcpyAsync(h, c->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return cuda_err(e);
}

// Friction factor C_f of Sec. 2.1 from the law's coefficient.
double friction_cf(int law, double g, double coef)
{
    switch (law) {
    case SWOF_FRIC_MANNING: return coef * coef;
    case SWOF_FRIC_STRICKLER: return 1.0 / (coef * coef);
    case SWOF_FRIC_DARCY: return coef / (8.0 * g);
    case SWOF_FRIC_CHEZY: return 1.0 / (coef * coef);
    default: return 0.0;
    }
}

// Tensor maps of the padded fields for the stage kernels' TMA ring: one
// 2-D map per field and tile width, the whole padded array (pitch x ny + 4
// elements) with a box of NTX columns x RING_ROWS rows; boxes reaching past
// the array are zero-filled.
template <typename T>
int make_sweep_maps(swof_ctx *c, Fields<T> &F)
{
    swof::EncodeTiledFn enc = swof::encode_tiled();
    if (!enc) return SWOF_ECUDA;
    const Params &P = c->P;
    T *fld[8] = {F.h, F.qx, F.qy, F.h1, F.qx1, F.qy1, c->prec == SWOF_FP64 ? F.z : F.dzx,
                 c->prec == SWOF_FP64 ? nullptr : F.dzy};
    const int widths[swof::N_MAP_WIDTHS] = {64, 128, 256};
    const CUtensorMapDataType dt =
        sizeof(T) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    cuuint64_t dims[2] = {(cuuint64_t)P.pitch, (cuuint64_t)(P.ny + 4)};
    cuuint64_t strides[1] = {(cuuint64_t)P.pitch * sizeof(T)};
    cuuint32_t es[2] = {1, 1};
    for (int w = 0; w < swof::N_MAP_WIDTHS; ++w) {
        std::memset(&c->tmaps[w], 0, sizeof c->tmaps[w]);
        cuuint32_t box[2] = {(cuuint32_t)widths[w], (cuuint32_t)swof::RING_ROWS};
        for (int f = 0; f < 8; ++f) {
            if (!fld[f]) continue;
            if (enc(&c->tmaps[w].m[f], dt, 2, (void *)fld[f], dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
                return SWOF_ECUDA;
        }
    }
    F.tmaps = c->tmaps;
    return SWOF_OK;
}

template <typename T>
int alloc_fields(swof_ctx *c, Fields<T> &F, const double *z, const swof_params *p)
{
    int st = SWOF_OK;
    size_t n = padded_elems(c);
    F.h = dalloc<T>(c, n, &st);
    F.qx = dalloc<T>(c, n, &st);
    F.qy = dalloc<T>(c, n, &st);
    F.h1 = dalloc<T>(c, n, &st);
    F.qx1 = dalloc<T>(c, n, &st);
    F.qy1 = dalloc<T>(c, n, &st);
    F.vinf = dalloc<T>(c, n, &st);
    c->nslots = c->L->slots(c->P);
    F.outflow_slots = dalloc<double>(c, (size_t)c->nslots, &st);
    F.infil_slots = dalloc<double>(c, (size_t)c->nslots, &st);
    if (st) return st;
    std::vector<double> zp = host_padded(c, z);
    const Params &P = c->P;
    if (c->prec == SWOF_FP64) {
        F.z = dalloc<T>(c, n, &st);
        if (st) return st;
        st = upload_padded<T>(c, F.z, zp);
    } else {
        // per-face differences, computed in FP64 then rounded
        std::vector<double> dzx(n, 0.0), dzy(n, 0.0);
        auto id = [&](int i, int j) { return (size_t)(j + 2) * P.pitch + (size_t)(i + P.lpad); };
        for (int j = 0; j < P.ny; ++j)
            for (int i = -2; i <= P.nx; ++i) dzx[id(i, j)] = zp[id(i + 1, j)] - zp[id(i, j)];
        for (int j = -2; j <= P.ny; ++j)
            for (int i = 0; i < P.nx; ++i) dzy[id(i, j)] = zp[id(i, j + 1)] - zp[id(i, j)];
        F.dzx = dalloc<T>(c, n, &st);
        F.dzy = dalloc<T>(c, n, &st);
        if (st) return st;
        st = upload_padded<T>(c, F.dzx, dzx);
        if (!st) st = upload_padded<T>(c, F.dzy, dzy);
    }
    if (st) return st;
    if (p->friction_map) {
        std::vector<double> cf((size_t)P.nx * P.ny);
        for (size_t k = 0; k < cf.size(); ++k) cf[k] = friction_cf(p->friction, p->g, p->friction_map[k]);
        F.cfmap = dalloc<T>(c, n, &st);
        if (!st) st = upload_interior<T>(c, F.cfmap, cf.data());
    }
    if (!st && p->ks_map) {
        F.ksmap = dalloc<T>(c, n, &st);
        if (!st) st = upload_interior<T>(c, F.ksmap, p->ks_map);
    }
    F.ctl = c->ctl;
    F.dt_seq = nullptr;
    F.dt_hist = nullptr;
    F.dt_hist_cap = 0;
    if (!st) st = make_sweep_maps<T>(c, F);
    return st;
}

void set_hist(swof_ctx *c)
{
    c->f64.dt_hist = c->dt_hist;
    c->f32.dt_hist = c->dt_hist;
    c->f64.dt_hist_cap = c->dt_cap;
    c->f32.dt_hist_cap = c->dt_cap;
    c->f64.dt_seq = c->dt_seq_n > 0 ? c->dt_seq : nullptr;
    c->f32.dt_seq = c->dt_seq_n > 0 ? c->dt_seq : nullptr;
    c->gen++;
}

// Make room in the dt history for `more` further steps.
int ensure_hist(swof_ctx *c, long long more)
{
    long long need = c->host_steps + more;
    if (need <= c->dt_cap) return SWOF_OK;
    long long cap = c->dt_cap ? c->dt_cap : 1024;
    while (cap < need) cap *= 2;
    double *p = nullptr;
    if (cudaMalloc(&p, (size_t)cap * sizeof(double)) != cudaSuccess) return SWOF_ENOMEM;
    cudaError_t e = cudaSuccess;
    if (c->dt_hist) {
        e = cudaMemcpyAsync(p, c->dt_hist, (size_t)c->dt_cap * sizeof(double), cudaMemcpyDeviceToDevice,
                            c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        cudaFree(c->dt_hist);
    }
    c->dt_hist = p;
    c->dt_cap = cap;
    set_hist(c);
    return cuda_err(e);
}

// Forget the partial wave-speed maximum a fused stage 2 left behind (the
// state or the tile shape changed): the next step runs the full pass.
int invalidate_lambda(swof_ctx *c)
{
    c->lam_valid = false;
    return cuda_err(cudaMemsetAsync(c->ctl->lam_bits, 0, sizeof c->ctl->lam_bits, c->stream));
}

// Tile-edge columns and rows of the current tile shape (plus the last
// column/row), whose wave speeds the ring kernel computes.
int update_rings(swof_ctx *c)
{
    const Params &P = c->P;
    int w = swof::TILE_SHAPES[P.tile_cfg2].ntx - 4, h = swof::TILE_SHAPES[P.tile_cfg2].h;
    std::vector<int> cols, rows;
    for (int i = 0; i < P.nx; ++i)
        if (i % w == 0 || i % w == w - 1 || i == P.nx - 1) cols.push_back(i);
    for (int j = 0; j < P.ny; ++j)
        if (j % h == 0 || j % h == h - 1 || j == P.ny - 1) rows.push_back(j);
    cudaError_t e = cudaMemcpyAsync(c->d_ring_cols, cols.data(), cols.size() * sizeof(int),
                                    cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->d_ring_rows, rows.data(), rows.size() * sizeof(int), cudaMemcpyHostToDevice,
                            c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    c->f64.ring_cols = c->f32.ring_cols = c->d_ring_cols;
    c->f64.ring_rows = c->f32.ring_rows = c->d_ring_rows;
    c->f64.n_ring_cols = c->f32.n_ring_cols = (int)cols.size();
    c->f64.n_ring_rows = c->f32.n_ring_rows = (int)rows.size();
    c->f64.ring_tw = c->f32.ring_tw = w;
    c->f64.ring_th = c->f32.ring_th = h;
    c->f64.ring_tgx = c->f32.ring_tgx = (P.nx + w - 1) / w;
    c->gen++;
    int st = cuda_err(e);
    return st ? st : invalidate_lambda(c);
}

}  // namespace

int swof_ctx_invalidate_lambda(swof_ctx *c) { return invalidate_lambda(c); }
int swof_ctx_ensure_hist(swof_ctx *c, long long more) { return ensure_hist(c, more); }

namespace {

// One step is three launches: wave speeds + dt (the full pass after a state
// change, else the tile-edge ring), then the two Heun stages.  First order:
// dt (from the speeds the previous step's end left; the full pass after a
// state change), the Euler stage, and its end (sources, ghosts, the speeds
// for the next dt).  With gauges, one more small launch records them.
int enqueue_steps(swof_ctx *c, int n)
{
    void *f = c->fields();
    const bool o1 = c->P.order == 1;
    // first order: the dt launch merges nothing of its own (empty ring)
    Fields<double> f64 = c->f64;
    Fields<float> f32 = c->f32;
    f64.n_ring_cols = f64.n_ring_rows = f32.n_ring_cols = f32.n_ring_rows = 0;
    void *fdt = o1 ? (c->prec == SWOF_FP64 ? (void *)&f64 : (void *)&f32) : f;
    int r = 0;
    c->launches_last = 0;
    auto first = [&]() {
        return c->lam_valid ? c->L->lambda_ring(c->P, fdt, c->stream) : c->L->lambda(c->P, f, c->stream);
    };
    auto s1 = [&]() { return o1 ? c->L->stage1_o1(c->P, f, c->stream) : c->L->stage1(c->P, f, c->stream); };
    auto s2 = [&]() { return o1 ? c->L->commit_o1(c->P, f, c->stream) : c->L->stage2(c->P, f, c->stream); };
    for (int s = 0; s < n && !r; ++s) {
        nvtxRangePushA("step");
        if (c->timing) {
            while ((int)c->ev.size() < c->ev_used + 4) {
                cudaEvent_t e;
                if (cudaEventCreate(&e) != cudaSuccess) return SWOF_ECUDA;
                c->ev.push_back(e);
            }
            cudaEventRecord(c->ev[c->ev_used + 0], c->stream);
            nvtxRangePushA("wave speeds + dt");
            r = first();
            nvtxRangePop();
            cudaEventRecord(c->ev[c->ev_used + 1], c->stream);
            nvtxRangePushA("stage 1");
            if (!r) r = s1();
            nvtxRangePop();
            cudaEventRecord(c->ev[c->ev_used + 2], c->stream);
            nvtxRangePushA("stage 2");
            if (!r) r = s2();
            nvtxRangePop();
            cudaEventRecord(c->ev[c->ev_used + 3], c->stream);
            c->ev_used += 4;
        } else {
            nvtxRangePushA("wave speeds + dt");
            r = first();
            nvtxRangePop();
            nvtxRangePushA("stage 1");
            if (!r) r = s1();
            nvtxRangePop();
            nvtxRangePushA("stage 2");
            if (!r) r = s2();
            nvtxRangePop();
        }
        if (!r && c->hmax) {
            r = c->L->hmax(c->P, f, c->stream);
            c->launches_last += 1;
        }
        if (!r && c->n_gauges > 0) {
            r = c->L->gauges(c->P, f, c->stream);
            c->launches_last += 1;
        }
        c->lam_valid = o1 || c->P.fuse_lambda != 0;
        c->launches_last += 3;
        nvtxRangePop();
    }
    return r ? SWOF_ECUDA : SWOF_OK;
}

// Every tile wet and processed: the state changed (or skipping starts).
int reset_activity(swof_ctx *c)
{
    if (!c->d_tile_act) return SWOF_OK;
    size_t nt = (size_t)c->nslots;
    cudaError_t e = cudaMemsetAsync(c->d_tile_act, 1, nt, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_tile_live, 1, nt, c->stream);
    return cuda_err(e);
}

bool all_finite(const double *a, size_t n)
{
    for (size_t k = 0; k < n; ++k)
        if (!std::isfinite(a[k])) return false;
    return true;
}

}  // namespace

extern "C" {

void swof_default_params(swof_params *p)
{
    if (!p) return;
    std::memset(p, 0, sizeof *p);
    p->g = 9.81;
    p->cfl = 0.5;
    p->h_dry = 1e-6;
    p->dt_max = 0.1;
    p->dt_min = 0.0;
    p->t_end = 1e30;
    p->precision = SWOF_FP64;
    p->cfl_mode = SWOF_CFL_SUM;
    p->friction = SWOF_FRIC_NONE;
}

int swof_create(int nx, int ny, double dx, double dy, const double *z, const swof_params *p, swof_ctx **out)
{
    if (!out) return SWOF_EINVAL;
    *out = nullptr;
    if (!z || !p || nx < 2 || ny < 2 || !(dx > 0) || !(dy > 0) || !std::isfinite(dx) || !std::isfinite(dy))
        return SWOF_EINVAL;
    if ((long long)nx * (long long)ny > (1LL << 33) || nx > (1 << 28) || ny > (1 << 25)) return SWOF_EINVAL;
    if (p->precision != SWOF_FP64 && p->precision != SWOF_FP32) return SWOF_EINVAL;
    if (p->cfl_mode != SWOF_CFL_SUM && p->cfl_mode != SWOF_CFL_MIN) return SWOF_EINVAL;
    if (p->friction < SWOF_FRIC_NONE || p->friction > SWOF_FRIC_CHEZY) return SWOF_EINVAL;
    if (p->friction != SWOF_FRIC_NONE && !p->friction_map &&
        !(std::isfinite(p->friction_coef) && p->friction_coef >= 0.0))
        return SWOF_EINVAL;
    if ((p->friction == SWOF_FRIC_STRICKLER || p->friction == SWOF_FRIC_CHEZY) && !p->friction_map &&
        !(p->friction_coef > 0.0))
        return SWOF_EINVAL;
    if (p->order != SWOF_ORDER_1 && p->order != SWOF_ORDER_2 && p->order != 2) return SWOF_EINVAL;
    for (int k = 0; k < 4; ++k) {
        if (p->bc[k] < SWOF_BC_WALL || p->bc[k] > SWOF_BC_IMPOSED_HQ) return SWOF_EINVAL;
        if (p->bc[k] >= SWOF_BC_IMPOSED_H &&
            !(std::isfinite(p->bc_h[k]) && p->bc_h[k] >= 0.0 && std::isfinite(p->bc_q[k]) && p->bc_q[k] >= 0.0))
            return SWOF_EINVAL;
    }
    if (!(p->g > 0) || !(p->cfl > 0) || !(p->h_dry >= 0) || !(p->dt_max > 0) || !(p->dt_min >= 0)) return SWOF_EINVAL;
    if (p->infiltration && !(p->dtheta > 0)) return SWOF_EINVAL;
    if (p->rain_rate < 0 || !(p->dt_fixed >= 0)) return SWOF_EINVAL;
    if (!all_finite(z, (size_t)nx * ny)) return SWOF_ENONFINITE;

    swof_ctx *c = new (std::nothrow) swof_ctx();
    if (!c) return SWOF_ENOMEM;
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        delete c;
        return SWOF_ECUDA;
    }
    c->prec = p->precision;
    c->esize = c->prec == SWOF_FP64 ? 8 : 4;
    c->L = c->prec == SWOF_FP64 ? &swof::launch_fp64() : &swof::launch_fp32();
    Params &P = c->P;
    P.nx = nx;
    P.ny = ny;
    P.lpad = 2;
    int align = 128 / (int)c->esize;
    P.pitch = ((P.lpad + nx + 2) + align - 1) / align * align;
    P.dx = dx;
    P.dy = dy;
    P.g = p->g;
    P.cfl = p->cfl;
    P.h_dry = p->h_dry == 0.0 ? 0.0 : p->h_dry;   // (-0 -> +0: the dry tests compare bit patterns)
    P.dt_max = p->dt_max;
    P.dt_min = p->dt_min;
    P.t_end = p->t_end;
    P.cfl_mode = p->cfl_mode;
    P.friction = p->friction;
    P.infiltration = p->infiltration ? 1 : 0;
    P.check_cfl = p->check_cfl ? 1 : 0;
    for (int k = 0; k < 4; ++k) {
        P.bc[k] = p->bc[k];
        P.bc_h[k] = p->bc_h[k];
        P.bc_q[k] = p->bc_q[k];
        P.fbc_h[k] = (float)p->bc_h[k];
        P.fbc_q[k] = (float)p->bc_q[k];
    }
    P.order = p->order == SWOF_ORDER_1 ? 1 : 2;
    P.cf = friction_cf(p->friction, p->g, p->friction_coef);
    P.rain_rate = p->rain_rate;
    P.rain_t_on = p->rain_t_on;
    P.rain_t_off = p->rain_t_off;
    P.ks = p->ks;
    P.psi = p->psi;
    P.dtheta = p->dtheta;
    P.dt_fixed = p->dt_fixed;
    P.area = dx * dy;
    P.fg = (float)P.g;
    P.fh_dry = (float)P.h_dry;
    P.fcf = (float)P.cf;
    P.fdx = (float)dx;
    P.fdy = (float)dy;
    P.fpsi = (float)P.psi;
    P.fdtheta = (float)P.dtheta;
    P.fks = (float)P.ks;
    P.fuse_lambda = 1;
    P.status = nullptr;           // set once the control block exists

    if (p->stream) {
        c->stream = (cudaStream_t)p->stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete c;
            return SWOF_ECUDA;
        }
        c->own_stream = true;
    }
    int st = cuda_err((cudaError_t)c->L->configure());
    if (!st) {
        c->ctl = dalloc<DevCtl>(c, 1, &st);
        if (!st) c->P.status = &c->ctl->status;
        c->d_red = dalloc<double>(c, 4 * 240, &st);
    }
    if (!st) st = c->prec == SWOF_FP64 ? alloc_fields<double>(c, c->f64, z, p) : alloc_fields<float>(c, c->f32, z, p);
    if (!st) {
        c->d_ring_cols = dalloc<int>(c, (size_t)nx, &st);
        c->d_ring_rows = dalloc<int>(c, (size_t)ny, &st);
    }
    if (!st) st = update_rings(c);
    if (!st) st = ensure_hist(c, 1024);
    if (!st) st = cuda_err(cudaStreamSynchronize(c->stream));
    if (st) {
        swof_destroy(c);
        return st;
    }
    *out = c;
    return SWOF_OK;
}

void swof_destroy(swof_ctx *c)
{
    if (!c) return;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    for (void *p : c->allocs) cudaFree(p);
    if (c->dt_seq) cudaFree(c->dt_seq);
    if (c->dt_hist) cudaFree(c->dt_hist);
    if (c->staging) cudaFree(c->staging);
    if (c->d_flag) cudaFree(c->d_flag);
    if (c->hmax) cudaFree(c->hmax);
    if (c->d_gauge_off) cudaFree(c->d_gauge_off);
    if (c->d_gauge_rec) cudaFree(c->d_gauge_rec);
    if (c->d_tile_act) cudaFree(c->d_tile_act);
    if (c->d_tile_live) cudaFree(c->d_tile_live);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    cudaSetDevice(dev);
    delete c;
}

static int clear_status(swof_ctx *c)
{
    return cuda_err(cudaMemsetAsync(&c->ctl->status, 0, sizeof c->ctl->status, c->stream));
}

__global__ void k_set_time(DevCtl *ctl, double t) { ctl->t = t; }

// Check a host state copied to the device: bit 1 of *flag for NaN/Inf,
// bit 2 for h < 0.
__global__ void k_check_state(const double *s, long long n, int *flag)
{
    int f = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < 3 * n; i += (long long)gridDim.x * blockDim.x) {
        const double v = s[i];
        if (!isfinite(v)) f |= 1;
        else if (i < n && v < 0.0) f |= 2;
    }
    f = __reduce_or_sync(0xffffffffu, f);
    if (f && (threadIdx.x & 31) == 0) atomicOr(flag, f);
}

// The staging buffer [3][ny][nx] of doubles and the flag word (allocated on
// first use, kept until destroy).
static int ensure_staging(swof_ctx *c)
{
    if (c->staging && c->d_flag) return SWOF_OK;
    const size_t n = (size_t)c->P.nx * c->P.ny;
    if (!c->staging && cudaMalloc(&c->staging, 3 * n * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        c->staging = nullptr;
        return SWOF_ENOMEM;
    }
    if (!c->d_flag && cudaMalloc(&c->d_flag, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        c->d_flag = nullptr;
        return SWOF_ENOMEM;
    }
    return SWOF_OK;
}

// Host arrays are copied to a device staging buffer (from pinned memory
// this is a plain DMA), checked there, and only then converted into the
// state: a rejected state leaves the old one untouched.
int swof_set_state(swof_ctx *c, const double *h, const double *hu, const double *hv)
{
    if (!c || !h || !hu || !hv) return SWOF_EINVAL;
    int st = ensure_staging(c);
    if (st) return st;
    const size_t n = (size_t)c->P.nx * c->P.ny;
    double *s0 = c->staging, *s1 = s0 + n, *s2 = s1 + n;
    cudaError_t e = cudaMemcpyAsync(s0, h, n * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s1, hu, n * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s2, hv, n * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_flag, 0, sizeof(int), c->stream);
    if (e != cudaSuccess) return SWOF_ECUDA;
    long long blocks = ((long long)(3 * n) + 255) / 256;
    k_check_state<<<(unsigned)(blocks < 152 * 16 ? (blocks > 0 ? blocks : 1) : 152 * 16), 256, 0, c->stream>>>(
        s0, (long long)n, c->d_flag);
    int flag = 0;
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, c->d_flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return SWOF_ECUDA;
    if (flag & 1) return SWOF_ENONFINITE;
    if (flag & 2) return SWOF_ENEGATIVE;
    st = cuda_err((cudaError_t)c->L->unpack(c->P, c->fields(), s0, s1, s2, SWOF_FP64, c->stream));
    if (!st) st = cuda_err((cudaError_t)c->L->ghosts(c->P, c->fields(), c->stream));
    if (!st) st = clear_status(c);
    if (!st) st = invalidate_lambda(c);
    if (!st) st = reset_activity(c);
    return st;
}

int swof_get_state(swof_ctx *c, double *h, double *hu, double *hv)
{
    if (!c || !h || !hu || !hv) return SWOF_EINVAL;
    int st = ensure_staging(c);
    if (st) return st;
    const size_t n = (size_t)c->P.nx * c->P.ny;
    double *s0 = c->staging, *s1 = s0 + n, *s2 = s1 + n;
    st = cuda_err((cudaError_t)c->L->pack(c->P, c->fields(), s0, s1, s2, SWOF_FP64, c->stream));
    if (st) return st;
    cudaError_t e = cudaMemcpyAsync(h, s0, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hu, s1, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hv, s2, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return SWOF_ECUDA;
    DevCtl d;
    st = read_ctl(c, &d);
    if (st) return st;
    return d.status;
}

int swof_set_state_device(swof_ctx *c, const void *h, const void *hu, const void *hv, int dtype)
{
    if (!c || !h || !hu || !hv || (dtype != SWOF_FP64 && dtype != SWOF_FP32)) return SWOF_EINVAL;
    int st = cuda_err((cudaError_t)c->L->unpack(c->P, c->fields(), h, hu, hv, dtype, c->stream));
    if (!st) st = cuda_err((cudaError_t)c->L->ghosts(c->P, c->fields(), c->stream));
    if (!st) st = clear_status(c);
    if (!st) st = invalidate_lambda(c);
    if (!st) st = reset_activity(c);
    return st;
}

int swof_get_state_device(swof_ctx *c, void *h, void *hu, void *hv, int dtype)
{
    if (!c || !h || !hu || !hv || (dtype != SWOF_FP64 && dtype != SWOF_FP32)) return SWOF_EINVAL;
    return cuda_err((cudaError_t)c->L->pack(c->P, c->fields(), h, hu, hv, dtype, c->stream));
}

int swof_get_infiltrated(swof_ctx *c, double *v)
{
    if (!c || !v) return SWOF_EINVAL;
    return c->prec == SWOF_FP64 ? download_interior<double>(c, c->f64.vinf, v)
                                : download_interior<float>(c, c->f32.vinf, v);
}

int swof_set_infiltrated(swof_ctx *c, const double *v)
{
    if (!c || !v) return SWOF_EINVAL;
    size_t n = (size_t)c->P.nx * c->P.ny;
    if (!all_finite(v, n)) return SWOF_ENONFINITE;
    for (size_t k = 0; k < n; ++k)
        if (v[k] < 0.0) return SWOF_ENEGATIVE;
    return c->prec == SWOF_FP64 ? upload_interior<double>(c, c->f64.vinf, v)
                                : upload_interior<float>(c, c->f32.vinf, v);
}

int swof_set_time(swof_ctx *c, double t)
{
    if (!c || !std::isfinite(t)) return SWOF_EINVAL;
    k_set_time<<<1, 1, 0, c->stream>>>(c->ctl, t);
    return cuda_err(cudaGetLastError());
}

// NVTX range over a scope (no-op unless a profiler is attached)
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

int swof_step(swof_ctx *c, int n, swof_step_info *info)
{
    NvtxRange range("swof_step");
    if (!c || n < 0) return SWOF_EINVAL;
    int st = ensure_hist(c, n);
    if (st) return st;
    c->ev_used = 0;
    if (n > 0) {
        if (c->use_graph && !c->timing) {
            if (!(c->gexec && c->graph_n == n && c->graph_gen == c->gen && c->graph_lam == c->lam_valid)) {
                if (c->gexec) cudaGraphExecDestroy(c->gexec);
                c->gexec = nullptr;
                cudaGraph_t g = nullptr;
                c->graph_lam = c->lam_valid;
                if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
                    return SWOF_ECUDA;
                int r = enqueue_steps(c, n);
                cudaError_t e = cudaStreamEndCapture(c->stream, &g);
                if (r || e != cudaSuccess) {
                    if (g) cudaGraphDestroy(g);
                    return SWOF_ECUDA;
                }
                cudaGraphExec_t ge = nullptr;      // kept only once it is valid
                e = cudaGraphInstantiate(&ge, g, 0);
                cudaGraphDestroy(g);
                if (e != cudaSuccess) return SWOF_ECUDA;
                c->gexec = ge;
                c->graph_n = n;
                c->graph_gen = c->gen;
            }
            if (cudaGraphLaunch(c->gexec, c->stream) != cudaSuccess) return SWOF_ECUDA;
            c->launches_last = (3 + (c->n_gauges > 0) + (c->hmax != nullptr)) * n;
            c->lam_valid = c->P.order == 1 || c->P.fuse_lambda != 0;
        } else {
            st = enqueue_steps(c, n);
            if (st) return st;
        }
        c->host_steps += n;
    }
    if (info) {
        DevCtl d;
        st = read_ctl(c, &d);
        if (st) return st;
        info->t = d.t;
        info->dt = d.last_dt;
        info->steps = d.steps;
        info->status = d.status;
        return d.status;
    }
    return SWOF_OK;
}

int swof_set_dt_sequence(swof_ctx *c, const double *dts, int n)
{
    if (!c || n < 0 || (n > 0 && !dts)) return SWOF_EINVAL;
    if (n > 0 && !all_finite(dts, (size_t)n)) return SWOF_ENONFINITE;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return SWOF_ECUDA;
    // the new sequence is complete on the device before the old one is
    // released: a call that fails leaves the replay as it was
    double *p = nullptr;
    if (n > 0) {
        if (cudaMalloc(&p, (size_t)n * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return SWOF_ENOMEM;
        }
        if (cudaMemcpy(p, dts, (size_t)n * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaFree(p);
            return SWOF_ECUDA;
        }
    }
    int v[2] = {0, n};
    cudaError_t e = cudaMemcpyAsync(&c->ctl->dt_seq_pos, v, sizeof v, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        if (p) cudaFree(p);
        return SWOF_ECUDA;
    }
    if (c->dt_seq) cudaFree(c->dt_seq);
    c->dt_seq = p;
    c->dt_seq_n = n;
    set_hist(c);
    return SWOF_OK;
}

int swof_get_dt_history(swof_ctx *c, double *out, int max, int *count)
{
    if (!c || !out || max < 0 || !count) return SWOF_EINVAL;
    DevCtl d;
    int st = read_ctl(c, &d);
    if (st) return st;
    long long n = d.steps < c->dt_cap ? d.steps : c->dt_cap;
    if (n > max) n = max;
    if (n > 0 && cudaMemcpy(out, c->dt_hist, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
        return SWOF_ECUDA;
    *count = (int)n;
    return SWOF_OK;
}

int swof_get_diagnostics(swof_ctx *c, swof_diag *d)
{
    if (!c || !d) return SWOF_EINVAL;
    int st = cuda_err((cudaError_t)c->L->reduce(c->P, c->fields(), c->d_red, c->nslots, c->stream));
    if (st) return st;
    std::vector<double> part(4 * 240);
    cudaError_t e = cudaMemcpyAsync(part.data(), c->d_red, part.size() * sizeof(double),
                                    cudaMemcpyDeviceToHost, c->stream);
    DevCtl ctl;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ctl, c->ctl, sizeof ctl, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return SWOF_ECUDA;
    double s = 0.0, mn = INFINITY, so = 0.0, si = 0.0;
    for (int b = 0; b < 240; ++b) {
        s += part[4 * b];
        mn = std::fmin(mn, part[4 * b + 1]);
        so += part[4 * b + 2];
        si += part[4 * b + 3];
    }
    d->t = ctl.t;
    d->last_dt = ctl.last_dt;
    d->steps = ctl.steps;
    d->volume = s * c->P.dx * c->P.dy;
    d->rain_in = ctl.rain_in;
    d->infiltrated = si * c->P.dx * c->P.dy;
    d->outflow = so;
    d->min_h = mn;
    d->cfl_viol = ctl.cfl_viol;
    return ctl.status;
}

int swof_enable_timing(swof_ctx *c, int on)
{
    if (!c) return SWOF_EINVAL;
    c->timing = on != 0;
    return SWOF_OK;
}

int swof_get_timing(swof_ctx *c, double *ms_l, double *ms_1, double *ms_2, int *launches)
{
    if (!c) return SWOF_EINVAL;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return SWOF_ECUDA;
    double a = 0, b = 0, d = 0;
    for (int k = 0; k + 3 < c->ev_used; k += 4) {
        float x = 0, y = 0, z = 0;
        cudaEventElapsedTime(&x, c->ev[k], c->ev[k + 1]);
        cudaEventElapsedTime(&y, c->ev[k + 1], c->ev[k + 2]);
        cudaEventElapsedTime(&z, c->ev[k + 2], c->ev[k + 3]);
        a += x;
        b += y;
        d += z;
    }
    if (ms_l) *ms_l = a;
    if (ms_1) *ms_1 = b;
    if (ms_2) *ms_2 = d;
    if (launches) *launches = c->launches_last;
    return SWOF_OK;
}

int swof_set_fp64_contraction(swof_ctx *c, int on)
{
    if (!c || c->prec != SWOF_FP64) return SWOF_EINVAL;
    const swof::Launch *L = on ? &swof::launch_fp64c() : &swof::launch_fp64();
    if (L == c->L) return SWOF_OK;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return SWOF_ECUDA;
    int st = cuda_err((cudaError_t)L->configure());
    if (st) return st;
    c->L = L;
    c->gen++;
    return SWOF_OK;
}

int swof_use_graph(swof_ctx *c, int on)
{
    if (!c) return SWOF_EINVAL;
    c->use_graph = on != 0;
    if (!on && c->gexec) {
        cudaStreamSynchronize(c->stream);
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    return SWOF_OK;
}

int swof_tile_shapes(int *ntx, int *rows, int max)
{
    for (int k = 0; k < swof::N_TILE_SHAPES && k < max; ++k) {
        if (ntx) ntx[k] = swof::TILE_SHAPES[k].ntx;
        if (rows) rows[k] = swof::TILE_SHAPES[k].h;
    }
    return swof::N_TILE_SHAPES;
}

int swof_set_tile_shape(swof_ctx *c, int shape)
{
    return swof_set_tile_shapes(c, shape, shape);
}

int swof_set_tile_shapes(swof_ctx *c, int shape1, int shape2)
{
    if (!c || shape1 < 0 || shape1 >= swof::N_TILE_SHAPES || shape2 < 0 || shape2 >= swof::N_TILE_SHAPES)
        return SWOF_EINVAL;
    if (c->skip_dry) shape1 = shape2;        // the tile flags need one tiling
    if (c->skip_dry && c->P.tile_cfg2 != shape2) {
        int st = reset_activity(c);
        if (st) return st;
    }
    c->P.tile_cfg = shape1;
    c->gen++;
    if (c->P.tile_cfg2 == shape2) return SWOF_OK;
    c->P.tile_cfg2 = shape2;
    return update_rings(c);
}

int swof_track_max_depth(swof_ctx *c, int on)
{
    if (!c) return SWOF_EINVAL;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return SWOF_ECUDA;
    if (c->hmax) cudaFree(c->hmax);
    c->hmax = nullptr;
    c->f64.hmax = nullptr;
    c->f32.hmax = nullptr;
    c->gen++;
    if (!on) return SWOF_OK;
    size_t bytes = padded_elems(c) * c->esize;
    if (cudaMalloc(&c->hmax, bytes) != cudaSuccess) {
        c->hmax = nullptr;
        return SWOF_ENOMEM;
    }
    const void *h = c->prec == SWOF_FP64 ? (const void *)c->f64.h : (const void *)c->f32.h;
    cudaError_t e = cudaMemcpyAsync(c->hmax, h, bytes, cudaMemcpyDeviceToDevice, c->stream);
    if (c->prec == SWOF_FP64) c->f64.hmax = (double *)c->hmax;
    else c->f32.hmax = (float *)c->hmax;
    return cuda_err(e);
}

int swof_get_max_depth(swof_ctx *c, double *out)
{
    if (!c || !out) return SWOF_EINVAL;
    if (!c->hmax) return SWOF_ESTATE;
    int st = ensure_staging(c);
    if (st) return st;
    const size_t n = (size_t)c->P.nx * c->P.ny;
    st = cuda_err((cudaError_t)c->L->pack1(c->P, c->hmax, c->staging, c->stream));
    if (st) return st;
    cudaError_t e = cudaMemcpyAsync(out, c->staging, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    return cuda_err(e);
}

int swof_set_gauges(swof_ctx *c, const int *cells, int n, int capacity)
{
    if (!c || n < 0 || (n > 0 && (!cells || capacity < 1))) return SWOF_EINVAL;
    const Params &P = c->P;
    std::vector<long long> off((size_t)n);
    for (int g = 0; g < n; ++g) {
        int i = cells[2 * g], j = cells[2 * g + 1];
        if (i < 0 || i >= P.nx || j < 0 || j >= P.ny) return SWOF_EINVAL;
        off[g] = (long long)(j + 2) * P.pitch + (i + P.lpad);
    }
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return SWOF_ECUDA;
    if (c->d_gauge_off) cudaFree(c->d_gauge_off);
    if (c->d_gauge_rec) cudaFree(c->d_gauge_rec);
    c->d_gauge_off = nullptr;
    c->d_gauge_rec = nullptr;
    c->n_gauges = 0;
    c->gauge_cap = 0;
    c->gen++;
    auto wire = [&](auto &F) {
        F.gauge_off = c->d_gauge_off;
        F.gauge_rec = c->d_gauge_rec;
        F.n_gauges = c->n_gauges;
        F.gauge_cap = c->gauge_cap;
    };
    // any failure below leaves the gauges off (nothing allocated, no offsets
    // for the kernel to read)
    auto drop = [&]() {
        if (c->d_gauge_off) cudaFree(c->d_gauge_off);
        if (c->d_gauge_rec) cudaFree(c->d_gauge_rec);
        c->d_gauge_off = nullptr;
        c->d_gauge_rec = nullptr;
    };
    cudaError_t e = cudaMemsetAsync(&c->ctl->gauge_n, 0, sizeof(long long), c->stream);
    int st = SWOF_OK;
    if (n > 0 && e == cudaSuccess) {
        if (cudaMalloc(&c->d_gauge_off, (size_t)n * sizeof(long long)) != cudaSuccess ||
            cudaMalloc(&c->d_gauge_rec, (size_t)capacity * (1 + 3 * (size_t)n) * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            drop();
            st = SWOF_ENOMEM;
        } else {
            e = cudaMemcpyAsync(c->d_gauge_off, off.data(), (size_t)n * sizeof(long long), cudaMemcpyHostToDevice,
                                c->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
            if (e == cudaSuccess) {
                c->n_gauges = n;
                c->gauge_cap = capacity;
            } else {
                drop();
            }
        }
    }
    wire(c->f64);
    wire(c->f32);
    return st != SWOF_OK ? st : cuda_err(e);
}

int swof_get_gauges(swof_ctx *c, double *out, int max_records, int *count)
{
    if (!c || !count || max_records < 0 || (max_records > 0 && !out)) return SWOF_EINVAL;
    DevCtl d;
    int st = read_ctl(c, &d);
    if (st) return st;
    long long n = c->n_gauges > 0 ? d.gauge_n : 0;
    if (n > max_records) n = max_records;
    if (n > 0 && cudaMemcpy(out, c->d_gauge_rec, (size_t)n * (1 + 3 * (size_t)c->n_gauges) * sizeof(double),
                            cudaMemcpyDeviceToHost) != cudaSuccess)
        return SWOF_ECUDA;
    *count = (int)n;
    return SWOF_OK;
}

int swof_set_dry_tile_skip(swof_ctx *c, int on)
{
    if (!c) return SWOF_EINVAL;
    if (on && c->P.order == 1) return SWOF_EINVAL;
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return SWOF_ECUDA;
    c->gen++;
    if (!on) {
        c->skip_dry = false;
        c->f64.tile_act = c->f32.tile_act = nullptr;
        c->f64.tile_live = c->f32.tile_live = nullptr;
        return SWOF_OK;
    }
    // both flag arrays or neither (a stage kernel reads both when skipping)
    if (!c->d_tile_act || !c->d_tile_live) {
        unsigned char *a = nullptr, *b = nullptr;
        if (cudaMalloc(&a, (size_t)c->nslots) != cudaSuccess || cudaMalloc(&b, (size_t)c->nslots) != cudaSuccess) {
            cudaGetLastError();
            if (a) cudaFree(a);
            return SWOF_ENOMEM;
        }
        if (c->d_tile_act) cudaFree(c->d_tile_act);
        if (c->d_tile_live) cudaFree(c->d_tile_live);
        c->d_tile_act = a;
        c->d_tile_live = b;
    }
    c->skip_dry = true;
    c->f64.tile_act = c->f32.tile_act = c->d_tile_act;
    c->f64.tile_live = c->f32.tile_live = c->d_tile_live;
    long long z[2] = {0, 0};
    cudaError_t e = cudaMemcpyAsync(&c->ctl->live_tiles, z, sizeof z, cudaMemcpyHostToDevice, c->stream);
    if (e != cudaSuccess) return SWOF_ECUDA;
    int st = reset_activity(c);
    if (!st) st = swof_set_tile_shapes(c, swof::SHALLOW_SHAPE, swof::SHALLOW_SHAPE);
    if (!st) st = cuda_err(cudaStreamSynchronize(c->stream));
    return st;
}

int swof_get_tile_activity(swof_ctx *c, long long *live, long long *tiles)
{
    if (!c || !live || !tiles) return SWOF_EINVAL;
    DevCtl d;
    int st = read_ctl(c, &d);
    if (st) return st;
    *live = d.live_tiles;
    *tiles = d.tiles;
    return SWOF_OK;
}

}  // extern "C"

namespace {

// Average ms of `reps` launches of one stage kernel with shape k (after one
// untimed launch).
int time_stage(swof_ctx *c, const Params &P0, void *fields, int stage, int k, int reps, cudaEvent_t e0,
               cudaEvent_t e1, double *out)
{
    Params P = P0;
    P.tile_cfg = k;
    P.tile_cfg2 = k;
    auto launch = [&]() {
        if (stage == 2) return c->L->stage2(P, fields, c->stream);
        return P.order == 1 ? c->L->stage1_o1(P, fields, c->stream) : c->L->stage1(P, fields, c->stream);
    };
    if (launch()) return SWOF_ECUDA;
    if (cudaEventRecord(e0, c->stream) != cudaSuccess) return SWOF_ECUDA;
    for (int r = 0; r < reps; ++r)
        if (launch()) return SWOF_ECUDA;
    if (cudaEventRecord(e1, c->stream) != cudaSuccess) return SWOF_ECUDA;
    float t = 0.0f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) return SWOF_ECUDA;
    *out = (double)t / reps;
    return SWOF_OK;
}

template <typename T>
int autotune_t(swof_ctx *c, Fields<T> &F, int reps, double *ms, int *best)
{
    // Stage 1 only reads U^n and writes U*: it is timed in place.  Stage 2
    // updates U^n and V_inf in place, so it is timed on scratch copies.
    Params P = c->P;
    P.no_budget = 1;
    P.check_cfl = 0;
    size_t n = padded_elems(c);
    std::vector<void *> scratch;
    int st = SWOF_OK;
    Fields<T> F1 = F;             // timed launches touch no output or tile flag
    F1.hmax = nullptr;
    F1.tile_act = F1.tile_live = nullptr;
    Fields<T> G = F1;
    for (T **dst : {&G.h, &G.qx, &G.qy, &G.vinf}) {
        void *p = nullptr;
        if (cudaMalloc(&p, n * sizeof(T)) != cudaSuccess) {
            st = SWOF_ENOMEM;
            break;
        }
        scratch.push_back(p);
        const T *src = (dst == &G.h) ? F.h : (dst == &G.qx) ? F.qx : (dst == &G.qy) ? F.qy : F.vinf;
        if (cudaMemcpyAsync(p, src, n * sizeof(T), cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
            st = SWOF_ECUDA;
        *dst = static_cast<T *>(p);
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (!st && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) st = SWOF_ECUDA;
    int bk[2] = {0, 0};
    for (int stage = 1; stage <= 2 && !st; ++stage) {
        double bms = INFINITY;
        for (int k = 0; k < swof::N_TILE_SHAPES && !st; ++k) {
            double m = 0.0;
            st = time_stage(c, P, stage == 1 ? (void *)&F1 : (void *)&G, stage, k, reps, e0, e1, &m);
            if (st) break;
            if (ms) ms[(stage - 1) * swof::N_TILE_SHAPES + k] = m;
            if (m < bms) {
                bms = m;
                bk[stage - 1] = k;
            }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamSynchronize(c->stream);
    for (void *p : scratch) cudaFree(p);
    if (st) return st;
    best[0] = bk[0];
    best[1] = bk[1];
    // the timed stage-2 launches added to the wave-speed words: start over
    st = swof_set_tile_shapes(c, bk[0], bk[1]);
    return st ? st : invalidate_lambda(c);
}

}  // namespace

extern "C" {

int swof_autotune(swof_ctx *c, int reps, double *ms, int *best)
{
    if (!c || reps < 1 || !best) return SWOF_EINVAL;
    return c->prec == SWOF_FP64 ? autotune_t<double>(c, c->f64, reps, ms, best)
                                : autotune_t<float>(c, c->f32, reps, ms, best);
}

const char *swof_strerror(int code)
{
    switch (code) {
    case SWOF_OK: return "ok";
    case SWOF_EINVAL: return "invalid argument";
    case SWOF_ENOMEM: return "device allocation failed";
    case SWOF_ECUDA: return "CUDA runtime error";
    case SWOF_ENONFINITE: return "non-finite value in the state or wave speeds";
    case SWOF_ENEGATIVE: return "negative water depth";
    case SWOF_ECFL: return "fixed dt exceeds the CFL bound";
    case SWOF_EDTSEQ: return "replayed dt sequence exhausted";
    case SWOF_ETIMEOUT: return "bounded device wait timed out";
    case SWOF_EDTUNDERFLOW: return "time step below dt_min";
    case SWOF_ESTATE: return "call not valid in this state";
    case SWOF_EBOUNDS: return "a kernel index check failed (debug build)";
    default: return "unknown status";
    }
}

const char *swof_version(void)
{
    return SWOF_BOUNDS_CHECK ? "libswof 0.2 debug (sm_103a; FP64 exact-order + FP32 bulk; index checks)"
                             : "libswof 0.2 (sm_103a; FP64 exact-order + FP32 bulk)";
}

int swof_debug_build(void) { return SWOF_BOUNDS_CHECK ? 1 : 0; }

int swof_debug_probe_index(swof_ctx *c, int i, int j)
{
    if (!c) return SWOF_EINVAL;
    if (!SWOF_BOUNDS_CHECK) return SWOF_ESTATE;
    if (c->L->probe(c->P, c->fields(), i, j, c->stream)) return SWOF_ECUDA;
    DevCtl d;
    int st = read_ctl(c, &d);
    return st ? st : d.status;
}

}  // extern "C"

// swof_ens_api.cu -- host side of the batched ensemble (include/swof.h,
// swof_ensemble_*): member contexts, the persistent-kernel work queue and
// its CUDA graph.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "swof_ctx.h"
#include "swof_ensemble.cuh"

namespace swof {
int launch_ensemble_fp32(const void *desc, int ntx, int grid, void *stream);
int launch_ensemble_fp64(const void *desc, int ntx, int grid, void *stream);
int ensemble_max_grid_fp32(int ntx, int *grid);
int ensemble_max_grid_fp64(int ntx, int *grid);
}  // namespace swof

struct swof_ens {
    int n = 0;
    int prec = SWOF_FP32;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<swof_ctx *> members;
    std::vector<int> mshape;             // per member: index into swof::ENS_SHAPES
    int ntx = 128;                       // the launch's CTA width (every member's shape has it)
    void *d_inst = nullptr;              // EnsInst<T>[n]
    long long *d_pre = nullptr;          // [3][n+1]
    unsigned int *d_done = nullptr;      // [n]
    swof::EnsQueue *d_q = nullptr;
    std::vector<long long> pre;
    long long phase_items[3] = {0, 0, 0};
    long long per_step = 0;
    long long spin_limit = 1LL << 22;
    int block_member = -1;
    int grid = 0;
    bool latched_timeout = false;
    // graph of one n-step launch (reset of the queue + the persistent kernel)
    cudaGraphExec_t gexec = nullptr;
    int graph_n = 0;
    unsigned long long graph_key = 0, key = 1;
    std::vector<unsigned> gens;          // member generations the descriptors were built from
};

namespace {

int cerr(cudaError_t e) { return e == cudaSuccess ? SWOF_OK : SWOF_ECUDA; }

template <typename T>
int build_desc(swof_ens *e, const Fields<T> &(*get)(swof_ctx *))
{
    const long long chunk = (long long)e->ntx * swof::RING_CHUNK_PER_THREAD;
    std::vector<swof::EnsInst<T>> inst((size_t)e->n);
    e->pre.assign(3 * (size_t)(e->n + 1), 0);
    for (int k = 0; k < e->n; ++k) {
        swof_ctx *c = e->members[k];
        const int ms = e->mshape[(size_t)k];
        const swof::TileShape sh = swof::ENS_SHAPES[ms];
        if (sh.ntx != e->ntx) return SWOF_EINVAL;
        const int W = sh.ntx - 4, H = sh.h;
        // the member's own tile shape: the same tiling, so its tile-edge
        // ring lists are the ones the launch's ring phase walks
        int st = swof_set_tile_shapes(c, swof::ENS_MEMBER_SHAPE[ms], swof::ENS_MEMBER_SHAPE[ms]);
        if (st) return st;
        swof::EnsInst<T> &I = inst[k];
        I.P = c->P;
        I.F = get(c);
        I.H = H;
        I.gdx = (c->P.nx + W - 1) / W;
        I.gdy = (c->P.ny + H - 1) / H;
        I.ring_cells = (long long)I.F.n_ring_cols * c->P.ny + (long long)I.F.n_ring_rows * c->P.nx;
        I.ring_chunks = (int)((I.ring_cells + chunk - 1) / chunk);
        long long items[3] = {I.ring_chunks, (long long)I.gdx * I.gdy, (long long)I.gdx * I.gdy};
        for (int p = 0; p < 3; ++p)
            e->pre[(size_t)p * (e->n + 1) + k + 1] = e->pre[(size_t)p * (e->n + 1) + k] + items[p];
    }
    e->gens.resize((size_t)e->n);
    for (int k = 0; k < e->n; ++k) e->gens[(size_t)k] = e->members[(size_t)k]->gen;
    e->per_step = 0;
    for (int p = 0; p < 3; ++p) {
        e->phase_items[p] = e->pre[(size_t)p * (e->n + 1) + e->n];
        e->per_step += e->phase_items[p];
    }
    cudaError_t r = cudaMemcpyAsync(e->d_inst, inst.data(), inst.size() * sizeof(inst[0]), cudaMemcpyHostToDevice,
                                    e->stream);
    if (r == cudaSuccess)
        r = cudaMemcpyAsync(e->d_pre, e->pre.data(), e->pre.size() * sizeof(long long), cudaMemcpyHostToDevice,
                            e->stream);
    if (r == cudaSuccess) r = cudaStreamSynchronize(e->stream);
    e->key++;
    return cerr(r);
}

const Fields<float> &get32(swof_ctx *c) { return c->f32; }
const Fields<double> &get64(swof_ctx *c) { return c->f64; }

int rebuild(swof_ens *e)
{
    return e->prec == SWOF_FP64 ? build_desc<double>(e, get64) : build_desc<float>(e, get32);
}

int max_grid(swof_ens *e)
{
    int g = 0;
    int r = e->prec == SWOF_FP64 ? swof::ensemble_max_grid_fp64(e->ntx, &g)
                                 : swof::ensemble_max_grid_fp32(e->ntx, &g);
    if (r) return SWOF_ECUDA;
    e->grid = g;
    return SWOF_OK;
}

// Enqueue one persistent launch advancing every member by n steps.
int enqueue(swof_ens *e, int n)
{
    cudaError_t r = cudaMemsetAsync(e->d_done, 0, (size_t)e->n * sizeof(unsigned int), e->stream);
    if (r == cudaSuccess) r = cudaMemsetAsync(e->d_q, 0, sizeof(swof::EnsQueue), e->stream);
    if (r != cudaSuccess) return SWOF_ECUDA;
    long long items = e->per_step * n;
    int grid = (int)(items < e->grid ? items : e->grid);
    if (grid < 1) grid = 1;
    if (e->prec == SWOF_FP64) {
        swof::EnsDesc<double> D{static_cast<const swof::EnsInst<double> *>(e->d_inst), e->n, e->d_pre,
                                {e->phase_items[0], e->phase_items[1], e->phase_items[2]}, e->per_step, n,
                                e->d_done, e->d_q, e->spin_limit, e->block_member};
        return swof::launch_ensemble_fp64(&D, e->ntx, grid, e->stream) ? SWOF_ECUDA : SWOF_OK;
    }
    swof::EnsDesc<float> D{static_cast<const swof::EnsInst<float> *>(e->d_inst), e->n, e->d_pre,
                           {e->phase_items[0], e->phase_items[1], e->phase_items[2]}, e->per_step, n,
                           e->d_done, e->d_q, e->spin_limit, e->block_member};
    return swof::launch_ensemble_fp32(&D, e->ntx, grid, e->stream) ? SWOF_ECUDA : SWOF_OK;
}

// Seed each member whose wave-speed words are not valid with the full
// reduction of its current state (no dt yet: the ring phase of the first
// step adds the ring cells, already counted, and computes dt).
int seed_lambda(swof_ens *e)
{
    for (swof_ctx *c : e->members) {
        if (c->lam_valid) continue;
        Params P = c->P;
        P.lam_partial = 1;
        if (c->L->lambda(P, c->fields(), c->stream)) return SWOF_ECUDA;
    }
    return SWOF_OK;
}

// Snapshot / restore of what a step changes in a member (autotuning).
struct Snap {
    std::vector<void *> bufs;
};

template <typename T>
int snap_t(swof_ctx *c, Fields<T> &F, Snap &s, bool restore)
{
    size_t n = (size_t)(c->P.ny + 4) * c->P.pitch;
    struct Item {
        void *p;
        size_t bytes;
    } items[] = {{F.h, n * sizeof(T)},
                 {F.qx, n * sizeof(T)},
                 {F.qy, n * sizeof(T)},
                 {F.vinf, n * sizeof(T)},
                 {F.outflow_slots, (size_t)c->nslots * sizeof(double)},
                 {F.infil_slots, (size_t)c->nslots * sizeof(double)},
                 {c->ctl, sizeof(DevCtl)}};
    const int ni = (int)(sizeof items / sizeof items[0]);
    if (!restore) {
        for (int k = 0; k < ni; ++k) {
            void *p = nullptr;
            if (cudaMalloc(&p, items[k].bytes) != cudaSuccess) return SWOF_ENOMEM;
            s.bufs.push_back(p);
            if (cudaMemcpyAsync(p, items[k].p, items[k].bytes, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess)
                return SWOF_ECUDA;
        }
    } else {
        for (int k = 0; k < ni && k < (int)s.bufs.size(); ++k)
            if (cudaMemcpyAsync(items[k].p, s.bufs[k], items[k].bytes, cudaMemcpyDeviceToDevice, c->stream) !=
                cudaSuccess)
                return SWOF_ECUDA;
    }
    return SWOF_OK;
}

int snap(swof_ctx *c, Snap &s, bool restore)
{
    return c->prec == SWOF_FP64 ? snap_t<double>(c, c->f64, s, restore) : snap_t<float>(c, c->f32, s, restore);
}

}  // namespace

extern "C" {

int swof_ensemble_create(int count, const swof_scenario *specs, const swof_params *common, swof_ens **out)
{
    if (!out) return SWOF_EINVAL;
    *out = nullptr;
    if (count < 1 || !specs || !common) return SWOF_EINVAL;
    if (common->precision != SWOF_FP64 && common->precision != SWOF_FP32) return SWOF_EINVAL;
    // the persistent kernel runs the second-order Heun step
    if (common->order == SWOF_ORDER_1) return SWOF_EINVAL;
    swof_ens *e = new (std::nothrow) swof_ens();
    if (!e) return SWOF_ENOMEM;
    e->n = count;
    e->mshape.assign((size_t)count, 0);
    e->ntx = swof::ENS_SHAPES[0].ntx;
    e->prec = common->precision;
    int st = SWOF_OK;
    if (common->stream) {
        e->stream = (cudaStream_t)common->stream;
    } else {
        st = cerr(cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking));
        e->own_stream = st == SWOF_OK;
    }
    for (int k = 0; k < count && !st; ++k) {
        const swof_scenario &sc = specs[k];
        if (!sc.z || !sc.h || !sc.hu || !sc.hv) {
            st = SWOF_EINVAL;
            break;
        }
        swof_params p = *common;
        p.friction_coef = sc.manning_n;
        p.friction = sc.manning_n > 0.0 ? SWOF_FRIC_MANNING : common->friction;
        p.rain_rate = sc.rain_rate;
        p.rain_t_on = sc.rain_t_on;
        p.rain_t_off = sc.rain_t_off;
        for (int b = 0; b < 4; ++b) {
            p.bc[b] = sc.bc[b];
            p.bc_h[b] = sc.bc_h[b];
            p.bc_q[b] = sc.bc_q[b];
        }
        p.friction_map = nullptr;
        p.ks_map = nullptr;
        p.stream = e->stream;
        swof_ctx *c = nullptr;
        st = swof_create(sc.nx, sc.ny, sc.dx, sc.dy, sc.z, &p, &c);
        if (st) break;
        e->members.push_back(c);
        st = swof_set_state(c, sc.h, sc.hu, sc.hv);
    }
    if (!st) {
        void *p = nullptr;
        size_t isz = e->prec == SWOF_FP64 ? sizeof(swof::EnsInst<double>) : sizeof(swof::EnsInst<float>);
        st = cerr(cudaMalloc(&p, isz * (size_t)count));
        e->d_inst = p;
        if (!st) st = cerr(cudaMalloc((void **)&e->d_pre, 3 * (size_t)(count + 1) * sizeof(long long)));
        if (!st) st = cerr(cudaMalloc((void **)&e->d_done, (size_t)count * sizeof(unsigned int)));
        if (!st) st = cerr(cudaMalloc((void **)&e->d_q, sizeof(swof::EnsQueue)));
    }
    if (!st) st = rebuild(e);
    if (!st) st = max_grid(e);
    if (st) {
        swof_ensemble_destroy(e);
        return st;
    }
    *out = e;
    return SWOF_OK;
}

void swof_ensemble_destroy(swof_ens *e)
{
    if (!e) return;
    if (e->stream) cudaStreamSynchronize(e->stream);
    if (e->gexec) cudaGraphExecDestroy(e->gexec);
    for (swof_ctx *c : e->members) swof_destroy(c);
    cudaFree(e->d_inst);
    cudaFree(e->d_pre);
    cudaFree(e->d_done);
    cudaFree(e->d_q);
    if (e->own_stream) cudaStreamDestroy(e->stream);
    delete e;
}

int swof_ensemble_size(const swof_ens *e) { return e ? e->n : 0; }

int swof_ensemble_member(swof_ens *e, int k, swof_ctx **ctx)
{
    if (!e || !ctx || k < 0 || k >= e->n) return SWOF_EINVAL;
    *ctx = e->members[(size_t)k];
    return SWOF_OK;
}

int swof_ensemble_step(swof_ens *e, int n, int *status)
{
    if (!e || n < 0) return SWOF_EINVAL;
    if (e->latched_timeout) return SWOF_ETIMEOUT;
    bool changed = false;
    for (size_t k = 0; k < e->members.size(); ++k) {
        swof_ctx *c = e->members[k];
        int st = swof_ctx_ensure_hist(c, n);
        if (st) return st;
        changed |= (c->gen != e->gens[k]);     // e.g. a dt sequence was set on a member
    }
    if (changed) {
        int st = rebuild(e);
        if (st) return st;
    }
    if (n > 0) {
        int st = seed_lambda(e);
        if (st) return st;
        if (e->gexec && e->graph_n == n && e->graph_key == e->key) {
            if (cudaGraphLaunch(e->gexec, e->stream) != cudaSuccess) return SWOF_ECUDA;
        } else {
            if (e->gexec) cudaGraphExecDestroy(e->gexec);
            e->gexec = nullptr;
            cudaGraph_t g = nullptr;
            if (cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return SWOF_ECUDA;
            int r = enqueue(e, n);
            cudaError_t ce = cudaStreamEndCapture(e->stream, &g);
            if (r || ce != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                return SWOF_ECUDA;
            }
            cudaGraphExec_t ge = nullptr;          // kept only once it is valid
            ce = cudaGraphInstantiate(&ge, g, 0);
            cudaGraphDestroy(g);
            if (ce != cudaSuccess) return SWOF_ECUDA;
            e->gexec = ge;
            e->graph_n = n;
            e->graph_key = e->key;
            if (cudaGraphLaunch(e->gexec, e->stream) != cudaSuccess) return SWOF_ECUDA;
        }
        for (swof_ctx *c : e->members) {
            c->lam_valid = true;
            c->host_steps += n;
        }
    }
    if (!status) return SWOF_OK;
    swof::EnsQueue q;
    if (cudaMemcpyAsync(&q, e->d_q, sizeof q, cudaMemcpyDeviceToHost, e->stream) != cudaSuccess ||
        cudaStreamSynchronize(e->stream) != cudaSuccess)
        return SWOF_ECUDA;
    if (q.abort) {
        e->latched_timeout = true;
        *status = SWOF_ETIMEOUT;
        return SWOF_ETIMEOUT;
    }
    *status = SWOF_OK;
    for (swof_ctx *c : e->members) {
        DevCtl d;
        if (cudaMemcpy(&d, c->ctl, sizeof d, cudaMemcpyDeviceToHost) != cudaSuccess) return SWOF_ECUDA;
        if (d.status) {
            *status = d.status;
            return d.status;
        }
    }
    return SWOF_OK;
}

int swof_ensemble_shapes(int *ntx, int *rows, int max)
{
    for (int k = 0; k < swof::N_ENS_SHAPES && k < max; ++k) {
        if (ntx) ntx[k] = swof::ENS_SHAPES[k].ntx;
        if (rows) rows[k] = swof::ENS_SHAPES[k].h;
    }
    return swof::N_ENS_SHAPES;
}

}  // extern "C"

namespace {

// Give the members the shapes ms (one launch width) and rebuild the launch.
int apply_shapes(swof_ens *e, const std::vector<int> &ms)
{
    const int ntx = swof::ENS_SHAPES[ms[0]].ntx;
    for (int s : ms)
        if (s < 0 || s >= swof::N_ENS_SHAPES || swof::ENS_SHAPES[s].ntx != ntx) return SWOF_EINVAL;
    if (ms == e->mshape && ntx == e->ntx) return SWOF_OK;
    e->mshape = ms;
    e->ntx = ntx;
    int st = rebuild(e);       // member tile shapes change: their ring words restart
    return st ? st : max_grid(e);
}

}  // namespace

extern "C" {

int swof_ensemble_set_shape(swof_ens *e, int shape)
{
    if (!e || shape < 0 || shape >= swof::N_ENS_SHAPES) return SWOF_EINVAL;
    return apply_shapes(e, std::vector<int>((size_t)e->n, shape));
}

int swof_ensemble_set_member_shape(swof_ens *e, int k, int shape)
{
    if (!e || k < 0 || k >= e->n || shape < 0 || shape >= swof::N_ENS_SHAPES) return SWOF_EINVAL;
    if (swof::ENS_SHAPES[shape].ntx != e->ntx) return SWOF_EINVAL;
    std::vector<int> ms = e->mshape;
    ms[(size_t)k] = shape;
    return apply_shapes(e, ms);
}

int swof_ensemble_get_member_shape(const swof_ens *e, int k)
{
    if (!e || k < 0 || k >= e->n) return SWOF_EINVAL;
    return e->mshape[(size_t)k];
}

int swof_ensemble_autotune(swof_ens *e, int steps, double *ms, int *best, int *member_shapes)
{
    if (!e || steps < 1 || !best) return SWOF_EINVAL;
    std::vector<Snap> snaps(e->members.size());
    int st = SWOF_OK;
    for (size_t k = 0; k < e->members.size() && !st; ++k) st = snap(e->members[k], snaps[k], false);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (!st && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) st = SWOF_ECUDA;
    long long hs = e->members.empty() ? 0 : e->members[0]->host_steps;
    // ms per step of `steps` steps with the member shapes ms_try; every
    // member is put back as it was afterwards
    auto timed = [&](const std::vector<int> &ms_try, double *out) -> int {
        int r = apply_shapes(e, ms_try);
        if (!r) r = seed_lambda(e);
        if (!r) r = cerr(cudaEventRecord(e0, e->stream));
        if (!r) r = enqueue(e, steps);
        if (!r) r = cerr(cudaEventRecord(e1, e->stream));
        float t = 0.0f;
        if (!r) r = cerr(cudaEventSynchronize(e1));
        if (!r) r = cerr(cudaEventElapsedTime(&t, e0, e1));
        swof::EnsQueue q;
        if (!r) r = cerr(cudaMemcpy(&q, e->d_q, sizeof q, cudaMemcpyDeviceToHost));
        if (!r && q.abort) r = SWOF_ETIMEOUT;
        for (size_t k = 0; k < e->members.size() && !r; ++k) {
            r = snap(e->members[k], snaps[k], true);
            e->members[k]->host_steps = hs;
        }
        if (!r) r = cerr(cudaStreamSynchronize(e->stream));
        *out = (double)t / steps;
        return r;
    };
    // member size classes (grid sides), in order of first appearance
    std::vector<std::pair<int, int>> cls;
    std::vector<int> of((size_t)e->n);
    for (int k = 0; k < e->n; ++k) {
        std::pair<int, int> sz(e->members[(size_t)k]->P.nx, e->members[(size_t)k]->P.ny);
        size_t c = 0;
        while (c < cls.size() && cls[c] != sz) ++c;
        if (c == cls.size()) cls.push_back(sz);
        of[(size_t)k] = (int)c;
    }
    // for each launch width: all members on its first shape, then per size
    // class each other height of that width, kept when the launch is faster
    const int widths[2] = {128, 64};
    double overall = INFINITY;
    std::vector<int> chosen = e->mshape;
    for (int wi = 0; wi < 2 && !st; ++wi) {
        std::vector<int> cand;
        for (int s = 0; s < swof::N_ENS_SHAPES; ++s)
            if (swof::ENS_SHAPES[s].ntx == widths[wi]) cand.push_back(s);
        std::vector<int> cur((size_t)e->n, cand[0]);
        double tcur = 0.0;
        st = timed(cur, &tcur);
        for (size_t c = 0; c < cls.size() && !st; ++c)
            for (size_t a = 1; a < cand.size() && !st; ++a) {
                std::vector<int> trial = cur;
                for (int k = 0; k < e->n; ++k)
                    if (of[(size_t)k] == (int)c) trial[(size_t)k] = cand[a];
                double t = 0.0;
                st = timed(trial, &t);
                if (!st && t < tcur) {
                    tcur = t;
                    cur = trial;
                }
            }
        if (st) break;
        if (ms) ms[wi] = tcur;
        if (tcur < overall) {
            overall = tcur;
            chosen = cur;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamSynchronize(e->stream);
    for (auto &s : snaps)
        for (void *p : s.bufs) cudaFree(p);
    if (st) return st;
    st = apply_shapes(e, chosen);
    // the restored control blocks hold the pre-tuning wave-speed words,
    // which are valid for the pre-tuning tiling only
    for (swof_ctx *c : e->members)
        if (!st) st = swof_ctx_invalidate_lambda(c);
    *best = e->mshape[0];
    if (member_shapes)
        for (int k = 0; k < e->n; ++k) member_shapes[k] = e->mshape[(size_t)k];
    return st;
}

int swof_ensemble_set_wait_limit(swof_ens *e, long long polls, int block_member)
{
    if (!e || polls < 1 || block_member < -1 || block_member >= e->n) return SWOF_EINVAL;
    e->spin_limit = polls;
    e->block_member = block_member;
    e->key++;
    return SWOF_OK;
}

}  // extern "C"

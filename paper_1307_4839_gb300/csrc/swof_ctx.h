// swof_ctx.h -- host-side context of libswof (internal; shared by the
// single-grid API and the ensemble API).
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "swof_internal.h"

using swof::DevCtl;
using swof::Fields;
using swof::Params;

struct swof_ctx {
    int device = 0;
    int prec = SWOF_FP64;
    size_t esize = 8;
    Params P{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    const swof::Launch *L = nullptr;
    Fields<double> f64{};
    Fields<float> f32{};
    std::vector<void *> allocs;
    DevCtl *ctl = nullptr;
    double *d_red = nullptr;
    int nslots = 0;
    double *dt_seq = nullptr;
    int dt_seq_n = 0;
    double *dt_hist = nullptr;
    long long dt_cap = 0;
    long long host_steps = 0;      // steps enqueued so far
    // CUDA graph of an n-step sequence
    bool use_graph = false;
    cudaGraphExec_t gexec = nullptr;
    int graph_n = 0;
    unsigned gen = 1, graph_gen = 0;
    // wave speeds: after a fused stage 2 the next step needs only the ring
    bool lam_valid = false;
    bool graph_lam = false;
    int *d_ring_cols = nullptr, *d_ring_rows = nullptr;
    // per-kernel timing of the last swof_step call
    bool timing = false;
    std::vector<cudaEvent_t> ev;
    int ev_used = 0;
    int launches_last = 0;
    // device staging of host state exchange: [3][ny][nx] doubles + a flag word
    double *staging = nullptr;
    int *d_flag = nullptr;
    // outputs along the run: running max depth, gauges; dry-tile flags
    void *hmax = nullptr;
    long long *d_gauge_off = nullptr;
    double *d_gauge_rec = nullptr;
    int n_gauges = 0;
    long long gauge_cap = 0;
    unsigned char *d_tile_act = nullptr, *d_tile_live = nullptr;
    bool skip_dry = false;
    // tensor maps of the padded fields for the stage kernels, per tile width
    swof::SweepMaps tmaps[swof::N_MAP_WIDTHS]{};

    void *fields() { return prec == SWOF_FP64 ? (void *)&f64 : (void *)&f32; }
};

// helpers implemented in swof_api.cu
int swof_ctx_invalidate_lambda(swof_ctx *c);
int swof_ctx_ensure_hist(swof_ctx *c, long long more);

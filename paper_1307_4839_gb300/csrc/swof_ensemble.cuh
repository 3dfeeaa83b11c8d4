// swof_ensemble.cuh -- one persistent kernel that advances a batch of
// independent shallow-water grids (uneven sizes, each with its own dt) by n
// time steps.
//
// Work is a queue of items ordered (step, phase, instance, tile) and handed
// out by one atomic counter; phases per step are
//   0: wave speeds of the instance's tile-edge ring + the dt control (the
//      tile interiors were reduced by the previous step's stage 2),
//   1: stage-1 sweep tiles, 2: stage-2 sweep tiles (swof_sweep.cuh).
// Before running an item a CTA waits until every earlier-phase item of the
// same instance has finished (a per-instance completion counter): items of
// different instances never wait on each other, so small grids run ahead
// while large ones are still busy.  No item waits on a later one and only
// running CTAs hold items, so the queue cannot deadlock whatever the number
// of resident CTAs.  Every wait is bounded: when it runs out the kernel
// latches an error flag that stops every CTA, and the host reads
// SWOF_ETIMEOUT.  The arithmetic per tile is exactly that of the
// single-grid kernels, so each member's results equal its own swof_step's.
//
// Compiled with -Xptxas -dlcm=cg: CTAs read data other CTAs wrote earlier in
// the same launch, so global loads must not be served from the non-coherent
// L1.
#pragma once
#include "swof_kernels.cuh"

namespace swof {

template <typename T>
struct EnsInst {
    Params P;
    Fields<T> F;
    int H;                     // rows per sweep tile of this instance (the launch fixes the width)
    int gdx, gdy;              // sweep tiling of this instance
    int ring_chunks;           // phase-0 items
    long long ring_cells;      // ring work (x-ring cells then y-ring cells)
};

struct EnsQueue {
    unsigned long long head;   // next item
    int abort;                 // set when a wait ran out
    int pad;
};

template <typename T>
struct EnsDesc {
    const EnsInst<T> *inst;
    int n;
    const long long *pre;      // [3][n+1] prefix sums of per-instance items per phase
    long long phase_items[3];  // items per phase in one step
    long long per_step;
    int steps;
    unsigned int *done;        // per-instance finished items
    EnsQueue *q;
    long long spin_limit;      // polls before a wait gives up
    int block_member;          // test hook: this member's waits never succeed (-1: off)
};

constexpr int RING_CHUNK_PER_THREAD = 8;

// Ring wave speeds for cells [c0, c1) of one instance; thread 0 of the last
// chunk runs the dt control.
template <typename T, int NTX>
__device__ __forceinline__ void ring_chunk(const EnsInst<T> &I, long long c0, long long c1,
                                           typename SweepSmem<T, NTX>::K *red)
{
    using K = typename SweepSmem<T, NTX>::K;
    const Params &P = I.P;
    const Fields<T> &F = I.F;
    DevCtl *ctl = F.ctl;
    if (ctl->status) return;
    const Scal<T> C = scal<T>(P);
    K kx = 0, ky = 0;
    const long long nxr = (long long)F.n_ring_cols * P.ny;
    for (long long k = c0 + threadIdx.x; k < c1; k += NTX) {
        if (k < nxr) {
            int gj = (int)(k / F.n_ring_cols), gi = F.ring_cols[k % F.n_ring_cols];
            V4<T> w = cell_rec(P, F, gi - 1, gj, C.hdry), m = cell_rec(P, F, gi, gj, C.hdry),
                  e = cell_rec(P, F, gi + 1, gj, C.hdry);
            kx = kmax(kx, speed_key(cell_speed(w.x, m.x, e.x, w.y, m.y, e.y, m.w, C.hdry, C.g)));
            // an imposed edge's boundary state (the ghost beside the edge cell)
            if (gi == 0 && P.bc[0] >= SWOF_BC_IMPOSED_H) kx = kmax(kx, speed_key(ab(w.y) + sq(C.g * w.x)));
            if (gi == P.nx - 1 && P.bc[1] >= SWOF_BC_IMPOSED_H) kx = kmax(kx, speed_key(ab(e.y) + sq(C.g * e.x)));
        } else {
            long long q = k - nxr;
            int gj = F.ring_rows[q / P.nx], gi = (int)(q % P.nx);
            V4<T> s_ = cell_rec(P, F, gi, gj - 1, C.hdry), m = cell_rec(P, F, gi, gj, C.hdry),
                  n = cell_rec(P, F, gi, gj + 1, C.hdry);
            ky = kmax(ky, speed_key(cell_speed(s_.x, m.x, n.x, s_.z, m.z, n.z, m.w, C.hdry, C.g)));
            if (gj == 0 && P.bc[2] >= SWOF_BC_IMPOSED_H) ky = kmax(ky, speed_key(ab(s_.z) + sq(C.g * s_.x)));
            if (gj == P.ny - 1 && P.bc[3] >= SWOF_BC_IMPOSED_H) ky = kmax(ky, speed_key(ab(n.z) + sq(C.g * n.x)));
        }
    }
    kx = block_max(kx, red);
    ky = block_max(ky, red + NTX / 32);
    if (threadIdx.x == 0) {
        atomicMax(&ctl->lam_bits[0], key64(kx));
        atomicMax(&ctl->lam_bits[1], key64(ky));
        __threadfence();
        if (atomicAdd(&ctl->done, 1u) == (unsigned int)I.ring_chunks - 1) control(P, F);
    }
}

__device__ __forceinline__ int find_inst(const long long *pre, int n, long long r)
{
    int lo = 0, hi = n;            // pre[lo] <= r < pre[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (pre[mid] <= r) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Four resident CTAs of 128 threads (eight of 64) per SM for FP32, registers
// capped at 128 without spills: on the 256-member batch (200 steps, default
// member shapes) 13.9 G cell-updates/s against 11.8 G at three CTAs (162
// registers; ncu: 0.72 eligible warps per cycle, issue 50 % busy) and 13.4 G
// at five (96 registers, spills); uncapped the stage code's live ranges take
// ~215 registers and two CTAs.
template <typename T>
constexpr int ens_min_blocks(int ntx)
{
    return std::is_same<T, float>::value ? (ntx == 128 ? 4 : (ntx == 64 ? 8 : 1)) : 1;
}

// The launch's CTAs are NTX wide; each member's tiles are NTX - 4 columns
// by its own H rows, from the heights the single-grid tile shapes have for
// that width (members of one launch may differ in H).
template <typename T, int STAGE, int NTX>
__device__ __forceinline__ void ens_sweep(const EnsInst<T> &I, int bx, int by, SweepSmem<T, NTX> &S)
{
    if constexpr (NTX == 64) {
        if (I.H == 16)
            sweep_tile<T, STAGE, NTX, 16, false>(I.P, I.F, bx, by, I.gdx, I.gdy, S);
        else
            sweep_tile<T, STAGE, NTX, 64, false>(I.P, I.F, bx, by, I.gdx, I.gdy, S);
    } else {
        if (I.H == 64)
            sweep_tile<T, STAGE, NTX, 64, false>(I.P, I.F, bx, by, I.gdx, I.gdy, S);
        else
            sweep_tile<T, STAGE, NTX, 32, false>(I.P, I.F, bx, by, I.gdx, I.gdy, S);
    }
}

template <typename T, int NTX>
__global__ void __launch_bounds__(NTX, ens_min_blocks<T>(NTX)) k_ensemble(EnsDesc<T> D)
{
    __shared__ SweepSmem<T, NTX> S;
    __shared__ long long s_local;
    __shared__ int s_inst, s_phase, s_go;
    const long long total = D.per_step * (long long)D.steps;
    for (;;) {
        if (threadIdx.x == 0) {
            int go = 0;
            long long it = (long long)atomicAdd(&D.q->head, 1ull);
            if (it < total && !*(volatile int *)&D.q->abort) {
                long long step = it / D.per_step, r = it % D.per_step;
                int phase = 0;
                while (phase < 2 && r >= D.phase_items[phase]) {
                    r -= D.phase_items[phase];
                    ++phase;
                }
                const long long *pre = D.pre + (size_t)phase * (D.n + 1);
                int i = find_inst(pre, D.n, r);
                long long local = r - pre[i];
                const long long ri = D.pre[i + 1] - D.pre[i];
                const long long si = D.pre[(D.n + 1) + i + 1] - D.pre[(D.n + 1) + i];
                unsigned long long need = (unsigned long long)step * (unsigned long long)(ri + 2 * si) +
                                          (phase >= 1 ? ri : 0) + (phase >= 2 ? si : 0);
                if (i == D.block_member) need += 1ull << 40;
                volatile unsigned int *dn = D.done + i;
                long long polls = 0;
                go = 1;
                while ((unsigned long long)*dn < need) {
                    if (*(volatile int *)&D.q->abort || ++polls > D.spin_limit) {
                        atomicExch(&D.q->abort, 1);
                        go = 0;
                        break;
                    }
                    __nanosleep(64);
                }
                __threadfence();
                s_local = local;
                s_inst = i;
                s_phase = phase;
            }
            s_go = go;
        }
        __syncthreads();
        if (!s_go) break;
        // by value: the compiler may then keep the scalars and pointers in
        // registers (a reference into global memory would be reloaded after
        // every store, as it could alias)
        const EnsInst<T> I = D.inst[s_inst];
        const long long local = s_local;
        if (s_phase == 0) {
            long long chunk = (long long)NTX * RING_CHUNK_PER_THREAD;
            long long c0 = local * chunk, c1 = c0 + chunk;
            if (c1 > I.ring_cells) c1 = I.ring_cells;
            ring_chunk<T, NTX>(I, c0, c1, &S.redk[0][0]);
        } else {
            int bx = (int)(local % I.gdx), by = (int)(local / I.gdx);
            if (s_phase == 1)
                ens_sweep<T, 1, NTX>(I, bx, by, S);
            else
                ens_sweep<T, 2, NTX>(I, bx, by, S);
        }
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) atomicAdd(D.done + s_inst, 1u);
    }
}

// Member tile shapes the ensemble kernel is built for, (threads, rows): the
// register-prefetch forms of single-grid shapes (ENS_MEMBER_SHAPE[k] is the
// index in TILE_SHAPES, which keeps a member's own tile-edge ring lists
// consistent with its ensemble tiling).  A launch takes one width.
constexpr int N_ENS_SHAPES = 4;
constexpr TileShape ENS_SHAPES[N_ENS_SHAPES] = {{128, 32}, {128, 64}, {64, 64}, {64, 16}};
constexpr int ENS_MEMBER_SHAPE[N_ENS_SHAPES] = {5, 6, 8, 9};

template <typename T>
int launch_ensemble_t(const EnsDesc<T> &D, int ntx, int grid, cudaStream_t s)
{
    if (ntx == 64)
        k_ensemble<T, 64><<<grid, 64, 0, s>>>(D);
    else
        k_ensemble<T, 128><<<grid, 128, 0, s>>>(D);
    return (int)cudaGetLastError();
}

template <typename T>
int ensemble_max_grid_t(int ntx, int *grid)
{
    int per_sm = 0;
    cudaError_t e = (ntx == 64) ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ensemble<T, 64>, 64, 0)
                                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ensemble<T, 128>, 128, 0);
    if (e != cudaSuccess) return (int)e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    *grid = (per_sm > 0 ? per_sm : 1) * sms;
    return 0;
}

}  // namespace swof

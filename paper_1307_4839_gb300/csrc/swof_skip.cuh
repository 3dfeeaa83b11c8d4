// swof_skip.cuh -- the tile-edge wave speeds when dry tiles are skipped
// (sm_103a).  (The stage kernels keep one CTA per tile: a wave of CTAs
// looping over tiles in a fixed stride was measured slower, because the
// wet region, long in y, then lands several live tiles on one CTA in turn.)
//
// The fused wave-speed pass of stage 2 covers each tile's interior; the
// speeds of every tile's first and last column (x) and first and last row
// (y) are left to a ring pass (Eq. (cfl): max over all cells).  With dry
// tiles skipped most tiles hold U^{n+1} = U^n = 0 and speeds 0, so this pass
// walks tiles instead of ring cells: one warp per tile, one byte read for a
// tile left alone, the ring of a processed tile otherwise.  The maximum is
// the same whatever the order, so dt is the flat ring pass's bit for bit.
#pragma once

SWOF_KERNELS_BEGIN

template <typename T>
__global__ void __launch_bounds__(256) k_lambda_ring_tiles(Params P, Fields<T> F)
{
    using K = decltype(speed_key(T(0)));
    __shared__ K red[2][NW];
    DevCtl *ctl = F.ctl;
    if (ctl->status) return;
    const Scal<T> C = scal<T>(P);
    const int W = F.ring_tw, H = F.ring_th, gx = F.ring_tgx, gy = (P.ny + H - 1) / H;
    const int ntiles = gx * gy;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    K kx = 0, ky = 0;
    for (int tile = blockIdx.x * (NT / 32) + warp; tile < ntiles; tile += gridDim.x * (NT / 32)) {
        if (!F.tile_live[tile]) continue;                 // warp-uniform
        const int bx = tile % gx, by = tile / gx;
        const int i0 = bx * W, i1 = min(i0 + W, P.nx) - 1;
        const int j0 = by * H, j1 = min(j0 + H, P.ny) - 1;
        // x speeds on the tile's first and last column
        for (int r = lane; r < 2 * (j1 - j0 + 1); r += 32) {
            const int gj = j0 + (r >> 1), gi = (r & 1) ? i1 : i0;
            V4<T> w = cell_rec(P, F, gi - 1, gj, C.hdry), m = cell_rec(P, F, gi, gj, C.hdry),
                  e = cell_rec(P, F, gi + 1, gj, C.hdry);
            if (!(is0(w.x) && is0(m.x) && is0(e.x)))   // three dry cells: speed 0
                    kx = kmax(kx, speed_key(cell_speed(w.x, m.x, e.x, w.y, m.y, e.y, m.w, C.hdry, C.g)));
            if (gi == 0 && P.bc[0] >= SWOF_BC_IMPOSED_H) kx = kmax(kx, speed_key(ab(w.y) + sq(C.g * w.x)));
            if (gi == P.nx - 1 && P.bc[1] >= SWOF_BC_IMPOSED_H) kx = kmax(kx, speed_key(ab(e.y) + sq(C.g * e.x)));
        }
        // y speeds on the tile's first and last row
        for (int c = lane; c < 2 * (i1 - i0 + 1); c += 32) {
            const int gi = i0 + (c >> 1), gj = (c & 1) ? j1 : j0;
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
        if (kx) atomicMax(&ctl->lam_bits[0], key64(kx));
        if (ky) atomicMax(&ctl->lam_bits[1], key64(ky));
        __threadfence();
        unsigned int ticket = atomicAdd(&ctl->done, 1u);
        if (ticket == gridDim.x - 1) control(P, F);
    }
}

// Ring pass of a step: by tiles when dry tiles are skipped (first order
// keeps the empty ring: its step end already reduced every speed).
template <typename T>
int launch_ring_t(const Params &P, void *f, void *stream)
{
    const Fields<T> &F = *static_cast<const Fields<T> *>(f);
    if (!F.tile_live || F.n_ring_cols + F.n_ring_rows == 0) return launch_lambda_ring_t<T>(P, f, stream);
    const int gy = (P.ny + F.ring_th - 1) / F.ring_th;
    const long long tiles = (long long)F.ring_tgx * gy;
    // two blocks per SM: each warp loops over tiles (a skipped one costs a
    // byte), and few blocks keep the completion-ticket atomics short
    long long b = (tiles + NT / 32 - 1) / (NT / 32);
    int grid = (int)(b < 152 * 2 ? (b > 0 ? b : 1) : 152 * 2);
    k_lambda_ring_tiles<T><<<grid, NT, 0, (cudaStream_t)stream>>>(P, F);
    return (int)cudaGetLastError();
}

SWOF_KERNELS_END

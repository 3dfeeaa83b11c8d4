// swof_sweep.cuh -- the Heun-stage kernel as a column sweep (sm_103a).
//
// A CTA of NTX threads owns NTX - 4 output columns (2 halo columns on each
// side) and H output rows.  Each thread owns one column and walks down the
// rows j0-2 .. j0+H+1 once:
//   * y direction: the column's last three rows live in registers, so the
//     y-reconstruction (Sec. 3.4), the y-face hydrostatic reconstruction +
//     HLL (Sec. 3.1, 3.3) and the update of row r-2 need no shared memory;
//     each y-face is computed once (the face above row r-2 becomes the face
//     below row r-1 in the next iteration);
//   * x direction: the current row goes through a one-row shared buffer
//     (3 barriers per row): x-reconstruction, then each thread's east face
//     flux, then its west neighbour's; the x flux differences of a row wait
//     two iterations in registers until that row is updated.
// Every input cell is read from HBM once, every output written once.  The
// stage kernels stage their input rows through a shared-memory ring filled
// by TMA: one thread issues, per block of RING_ROWS rows, one 2-D tensor
// copy per field (NTX columns x RING_ROWS rows, zero-filled outside the
// array) several blocks ahead, completion on one mbarrier per slot, so the
// bytes in flight depend neither on the registers a thread holds nor on
// per-thread address work.  (The persistent ensemble kernel keeps a
// one-row register prefetch.)
// The per-cell arithmetic is exactly the one of the oracle (same functions,
// same operation order), so the FP64 instantiation stays bit-identical to
// it; work whose result is known exactly is skipped (each case below says
// why the skipped value is the one the full path gives): the x part of a
// row dry across the CTA, a thread's x reconstruction and east face when
// its cells are dry, the y part of a column window of three dry cells, the
// update of a dry cell whose fluxes are all +0, and the wave speeds of dry
// cell triples.  Dry tests run on bit patterns, off GB300's narrow FP64 pipe.
#pragma once

SWOF_KERNELS_BEGIN

template <typename T>
struct Cell {
    T h, u, v, rh, qx, qy, zy;
};

template <typename T>
__device__ __forceinline__ Cell<T> make_cell(T h, T qx, T qy, T zy, T hdry)
{
    Cell<T> c = {h, T(0), T(0), T(0), qx, qy, zy};
    if (gt_pos(h, hdry)) {
        c.rh = rcp(h);
        c.u = qx * c.rh;
        c.v = qy * c.rh;
    }
    return c;
}

// CTA-wide barrier / AND-vote; a one-warp CTA needs only the warp's own
// (memory-ordering) synchronisation.
template <int NTX>
__device__ __forceinline__ void cta_sync()
{
    if constexpr (NTX == 32)
        __syncwarp();
    else
        __syncthreads();
}
template <int NTX>
__device__ __forceinline__ int cta_and(int p)
{
    if constexpr (NTX == 32) {
        __syncwarp();
        return __all_sync(0xffffffffu, p);
    } else {
        return __syncthreads_and(p);
    }
}

__device__ __forceinline__ unsigned long long bits(double x) { return (unsigned long long)__double_as_longlong(x); }
__device__ __forceinline__ unsigned int bits(float x) { return __float_as_uint(x); }

// FP32 depth update with stochastic rounding.  The stored depth of a deep
// cell changes each step by a near-constant amount of the order of one float
// ulp (the rain of one step, a pool draining evenly); rounded to nearest,
// that increment is lost or rounded up the same way every step, and cells in
// different binades drift apart -- a bias growing with the number of steps
// (relative L1 against FP64 up to 1.5e-5 in h and 4e-5 in hu over 1000 steps
// of the ensemble's rain-on-reservoir members).  Here a + b is rounded to the
// neighbouring float on the side of its exact value with probability
// |error| / spacing, so the rounding is unbiased on average and the error
// grows like a random walk instead.  The exact error comes from TwoSum
// (Knuth); the random bits from Chris Wellons' "lowbias32" integer hash
// (hash-prospector, 2018) of the cell's index in the grid and the step's
// simulated time t (hashed once per launch into ts): the same state at the
// same time gives the same result whatever the step count, tiling or
// context, and every cell draws afresh at every step.  (The operands' bits in
// place of the cell index made equal cells of a pool round alike, so a whole
// pool's rounding errors added up: 10x the error on one ensemble member.)
__device__ __forceinline__ unsigned lowbias32(unsigned x)
{
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}
__device__ __forceinline__ float sr_add(float a, float b, unsigned cell, unsigned ts)
{
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);          // a + b = s + e exactly
    if (!(s > 0.0f) || e == 0.0f) return s;             // no neighbour below +0 to take
    const unsigned sb = __float_as_uint(s);
    const float nb = __uint_as_float(e > 0.0f ? sb + 1u : sb - 1u);   // neighbour on e's side
    const float gap = fabsf(nb - s);
    const unsigned u = lowbias32(cell ^ ts);
    return (float)(u >> 8) * 0x1p-24f * gap < fabsf(e) ? nb : s;
}

// TMA input ring: ring_depth<T, NTX>() slots of RING_ROWS rows; a slot holds
// the fields of the stage input (h, qx, qy, then z (FP64) or dz_x, dz_y
// (FP32)) and, in stage 2, U^n (h, qx, qy) of the rows two above, each
// field a [RING_ROWS][NTX] block (128-byte aligned for the tensor copy).
constexpr int RING_MAX_SLOTS = 4;
template <typename T, int STAGE>
constexpr int ring_fields()
{
    return (std::is_same<T, double>::value ? 4 : 5) + (STAGE == 2 ? 3 : 0);
}
// slots: as many blocks (2..4) as fit in RING_CAP bytes, so several CTAs
// share an SM (FP64: a smaller ring and more resident warps to cover the
// FP64 pipe's latency)
#ifndef SWOF_RING_CAP64
#define SWOF_RING_CAP64 (32 * 1024)
#endif
template <typename T, int STAGE, int NTX>
constexpr int ring_depth()
{
    constexpr size_t blk = (size_t)ring_fields<T, STAGE>() * RING_ROWS * NTX * sizeof(T);
    constexpr size_t cap = std::is_same<T, double>::value ? SWOF_RING_CAP64 : 56 * 1024;
    constexpr size_t d = cap / blk;
    return d < 2 ? 2 : (d > RING_MAX_SLOTS ? RING_MAX_SLOTS : (int)d);
}
template <typename T, int STAGE, int NTX>
constexpr size_t ring_bytes()
{
    return (size_t)ring_depth<T, STAGE, NTX>() * ring_fields<T, STAGE>() * RING_ROWS * NTX * sizeof(T);
}
// bounded mbarrier wait of the ring: false when the limit ran out
__device__ __forceinline__ bool ring_wait(uint32_t bar, uint32_t parity)
{
    for (int i = 0; i < (1 << 20); ++i)
        if (tc05::mbar_try_wait(bar, parity)) return true;
    return false;
}

template <typename T, int NTX>
struct SweepSmem {
    using K = decltype(speed_key(T(0)));
    V4<T> st[NTX];        // {h, u, v, 1/h} of the current row
    T zx[NTX];            // FP64: z; FP32: dz_x
    V4<T> m[NTX];         // x-recon minus side {h, z, u, v}
    V4<T> f[NTX];         // flux through the cell's east face
    V4<T> nw[2][NTX];     // U^{n+1} {h, u, v, 1/h} of the finished row
    double red[NTX / 32];
    K redk[2][NTX / 32];
    int flag;             // dry-tile skipping: bit 0 live now, bit 1 live last step
    unsigned long long bar[RING_MAX_SLOTS];   // TMA ring: one mbarrier per slot
};

// One stage over the tile (bx, by) of a (gdx x gdy) tiling; the kernel
// below maps it to its block index, the ensemble kernel to a queue item.
// DRY_SKIP: let a CTA skip the x part of a row (and the wave speeds of three
// rows) that is dry across its columns -- exact, and a large saving on
// mostly dry grids; grids that are wet everywhere (the ensemble's rain
// scenarios) run without the vote.
// ORD1: the first-order stage (Sec. 3.3): face values = cell values.
// TMA_RING: stage the input rows through the TMA ring (ring != nullptr,
// tensor maps M); else a one-row register prefetch.
// With F.tile_act set (dry-tile skipping), a tile whose 3x3 tile
// neighbourhood held no water after the last step, with no rain and no
// imposed edge, is left alone: every flux of the step is exactly zero there
// and U^{n+1} = U^n (stage 2 works in place); stage 1 writes its U* = 0 once
// when the tile turns dry, for the neighbours' halos.
template <typename T, int STAGE, int NTX, int H, bool DRY_SKIP = true, bool ORD1 = false, bool TMA_RING = false>
__device__ __forceinline__ void sweep_tile(const Params &P, const Fields<T> &F, int bx, int by, int gdx, int gdy,
                                           SweepSmem<T, NTX> &S, T *ring = nullptr, const SweepMaps *M = nullptr)
{
    constexpr bool fp64 = std::is_same<T, double>::value;
    constexpr int W = NTX - 4;
    constexpr int NF = ring_fields<T, STAGE>();
    constexpr int RD = ring_depth<T, STAGE, NTX>();
    constexpr int RR = RING_ROWS;
    static_assert(RD >= 2 && RD <= RING_MAX_SLOTS && (RR & (RR - 1)) == 0, "ring shape");
    constexpr int FH = 0, FQX = 1, FQY = 2, FZX = 3, FZY = 4, FUN = fp64 ? 4 : 5;
    using K = decltype(speed_key(T(0)));
    V4<T> *s_st = S.st;
    T *s_zx = S.zx;
    V4<T> *s_m = S.m;
    V4<T> *s_f = S.f;
    double *s_red = S.red;

    const DevCtl *ctl = F.ctl;
    if (ctl->status) return;
    const Scal<T> C = scal<T>(P);
    const int t = threadIdx.x;
    const int gi = bx * W - 2 + t;
    const int j0 = by * H;
    const int blk = by * gdx + bx;
    const bool col_in = gi <= P.nx + 1;
    const bool out_col = t >= 2 && t < NTX - 2 && gi < P.nx;
    bool dead = false;
    if (F.tile_act) {
        if (STAGE == 1) {
            if (t == 0) {
                int live = ctl->rain_active != 0;
                live |= (bx == 0 && P.bc[0] >= SWOF_BC_IMPOSED_H) || (bx == gdx - 1 && P.bc[1] >= SWOF_BC_IMPOSED_H) ||
                        (by == 0 && P.bc[2] >= SWOF_BC_IMPOSED_H) || (by == gdy - 1 && P.bc[3] >= SWOF_BC_IMPOSED_H);
                for (int dj = -1; dj <= 1; ++dj)
                    for (int di = -1; di <= 1; ++di) {
                        int a = bx + di, b = by + dj;
                        if (a >= 0 && a < gdx && b >= 0 && b < gdy) live |= F.tile_act[b * gdx + a];
                    }
                int was = F.tile_live[blk];
                F.tile_live[blk] = (unsigned char)live;
                S.flag = live | (was << 1);
                if (live) atomicAdd((unsigned long long *)&F.ctl->live_tiles, 1ull);
                if (blk == 0) atomicAdd((unsigned long long *)&F.ctl->tiles, (unsigned long long)(gdx * gdy));
            }
            cta_sync<NTX>();
            const int fl = S.flag;
            dead = !(fl & 1);
            if (dead && (fl & 2) && out_col)      // turned dry: its U* is 0 from now on
                for (int ro = j0; ro < j0 + H && ro < P.ny; ++ro)
                    store_cell<T, false>(P, F.h1, F.qx1, F.qy1, gi, ro, T(0), T(0), T(0));
        } else {
            dead = F.tile_live[blk] == 0;
        }
    }
    const T *hin = (STAGE == 1) ? F.h : F.h1;
    const T *qxin = (STAGE == 1) ? F.qx : F.qx1;
    const T *qyin = (STAGE == 1) ? F.qy : F.qy1;
    T dt, dtdx, dtdy, rdt;
    if constexpr (fp64) {
        dt = ctl->dt; dtdx = ctl->dtdx; dtdy = ctl->dtdy; rdt = ctl->rdt;
    } else {
        dt = ctl->fdt; dtdx = ctl->fdtdx; dtdy = ctl->fdtdy; rdt = ctl->frdt;
    }
    const bool rain = ctl->rain_active != 0;
    unsigned sr_ts = 0;                                  // FP32 depth rounding: the step's time, hashed
    if constexpr (!fp64 && STAGE == 2) {
        const unsigned long long tb = (unsigned long long)__double_as_longlong(ctl->t);
        sr_ts = lowbias32((unsigned)tb ^ lowbias32((unsigned)(tb >> 32) + 0x9e3779b9u));
    }
    const T hg = T(0.5) * C.g;
    const T cdx = fp64 ? T(P.dx) : T(P.fdx), cdy = fp64 ? T(P.dy) : T(P.fdy);   // (no FP64 conversion per row)

    // row loader (zeros outside the padded array)
    auto load = [&](int r, T &h, T &qx, T &qy, T &zx, T &zy) {
        h = qx = qy = zx = zy = T(0);
        if (col_in && r <= P.ny + 1) {
            size_t o = pidx(P, gi, r);
            h = hin[o];
            qx = qxin[o];
            qy = qyin[o];
            if constexpr (fp64) {
                zx = F.z[o];
                zy = zx;
            } else {
                zx = F.dzx[o];
                zy = F.dzy[o];
            }
        }
    };
    // TMA ring: block b holds grid rows j0 - 2 + b*RR .. + RR - 1 of the
    // stage input and U^n of the rows two above; thread 0 issues it.  The
    // tile's first column sits on a 16-byte boundary (lpad = 2 and W a
    // multiple of 4), as a tensor copy needs.
    const int nblk = (H + 4 + RR - 1) / RR;
    const int x0 = bx * W - 2 + P.lpad;
    auto issue_block = [&](int b) {
        if (b >= nblk) return;
        // a tensor copy starts on a 16-byte boundary
        if (!bounds_ok(P, (x0 * (int)sizeof(T)) % 16 == 0 && b >= 0)) return;
        const int sl = b % RD;
        const uint32_t bar = tc05::smem_u32(&S.bar[sl]);
        T *base = ring + sl * (NF * RR * NTX);
        const int y0 = j0 + b * RR;                 // padded row of grid row j0 - 2 + b*RR
        tc05::mbar_arrive_expect_tx(bar, (uint32_t)(NF * RR * NTX * sizeof(T)));
        const int in0 = STAGE == 1 ? 0 : 3;         // U^n (h, qx, qy) or U* (h1, qx1, qy1)
        tc05::tma_load_2d(tc05::smem_u32(base + FH * RR * NTX), &M->m[in0 + 0], x0, y0, bar);
        tc05::tma_load_2d(tc05::smem_u32(base + FQX * RR * NTX), &M->m[in0 + 1], x0, y0, bar);
        tc05::tma_load_2d(tc05::smem_u32(base + FQY * RR * NTX), &M->m[in0 + 2], x0, y0, bar);
        tc05::tma_load_2d(tc05::smem_u32(base + FZX * RR * NTX), &M->m[6], x0, y0, bar);
        if constexpr (!fp64) tc05::tma_load_2d(tc05::smem_u32(base + FZY * RR * NTX), &M->m[7], x0, y0, bar);
        if constexpr (STAGE == 2) {
            tc05::tma_load_2d(tc05::smem_u32(base + (FUN + 0) * RR * NTX), &M->m[0], x0, y0 - 2, bar);
            tc05::tma_load_2d(tc05::smem_u32(base + (FUN + 1) * RR * NTX), &M->m[1], x0, y0 - 2, bar);
            tc05::tma_load_2d(tc05::smem_u32(base + (FUN + 2) * RR * NTX), &M->m[2], x0, y0 - 2, bar);
        }
    };
    // a row of the ring (field f at rowp[f * RR * NTX])
    auto ring_row = [&](int kk) -> const T * {
        if (!bounds_ok(P, kk >= 0 && kk < H + 4)) kk = 0;
        return ring + ((kk / RR) % RD) * (NF * RR * NTX) + (kk & (RR - 1)) * NTX + t;
    };
    bool ring_ok = true;

    Cell<T> ra{}, rb{};                 // rows r-2, r-1
    V4<T> ypa{};                        // y-recon plus side of row r-2 {h, z, v, u}
    T fcya = T(0);                      // centred y source term of row r-2
    V4<T> gs{};                         // y-face flux below row r-2
    T a1q[2] = {T(0), T(0)}, a2q[2] = {T(0), T(0)}, a3q[2] = {T(0), T(0)};  // x parts, rows r-1, r
    T outacc = T(0), infacc = T(0);
    K k2x = 0, k2y = 0;
    K lx = 0, ly = 0;                   // wave speeds of U^{n+1} (stage 2, fused)
    T y1h = T(0), y1v = T(0), y1rh = T(0), y2h = T(0), y2v = T(0);   // U^{n+1} rows ro-1, ro-2
    const bool xlam = t >= 3 && t <= NTX - 4 && gi <= P.nx - 2;

    // per-cell data of the row updated in the next iteration, fetched one
    // iteration ahead: U^n (stage 2; from the ring when there is one), the
    // C_f map, V_inf and K_s
    T un_h = T(0), un_qx = T(0), un_qy = T(0), pn2 = C.cf, pvi = T(0), pks = C.ks;
    const bool want_prefetch = (STAGE == 2 && (!TMA_RING || P.infiltration)) || F.cfmap != nullptr;
    auto prefetch = [&](int ro) {
        if (!want_prefetch || !(out_col && ro >= j0 && ro < j0 + H && ro < P.ny)) return;
        size_t o = pidx(P, gi, ro);
        if (STAGE == 2) {
            if (!TMA_RING) {
                un_h = F.h[o];
                un_qx = F.qx[o];
                un_qy = F.qy[o];
            }
            if (P.infiltration) {
                pvi = F.vinf[o];
                if (F.ksmap) pks = F.ksmap[o];
            }
        }
        if (F.cfmap) pn2 = F.cfmap[o];
    };

    bool anywet = false;                // a row of U^{n+1} of this tile holds water (stage 2, uniform)
    int dryrun = 0;                     // consecutive rows voted dry (ring path)
    if (!dead) {
    T nh, nqx, nqy, nzx, nzy;
    if constexpr (TMA_RING) {
        if (t == 0) {
#pragma unroll
            for (int sl = 0; sl < RD; ++sl) tc05::mbar_init(tc05::smem_u32(&S.bar[sl]), 1);
            asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        }
        cta_sync<NTX>();
        if (t == 0)
            for (int b = 0; b < RD - 1; ++b) issue_block(b);
    } else {
        load(j0 - 2, nh, nqx, nqy, nzx, nzy);
    }
    // ring: wait for the block of row kk when kk starts it
    auto ring_arrive = [&](int kk) {
        if ((kk & (RR - 1)) == 0) {
            const int b = kk / RR;
            if (!ring_wait(tc05::smem_u32(&S.bar[b % RD]), (uint32_t)((b / RD) & 1))) ring_ok = false;
        }
    };
    // U^n of the row updated at row kk (zeros outside the tile, as the
    // register path reads them)
    auto un_ok = [&](int kk) {
        const int ro = j0 - 4 + kk;
        return out_col && ro >= j0 && ro < j0 + H && ro < P.ny;
    };
    // The register path walks two rows per trip, so the register window
    // rotates by renaming instead of moves (measured ~1.5 % per stage).
    // The ring path walks one: its dry runs move k inside the trip.
    constexpr int UNROLL = (DRY_SKIP && !TMA_RING) ? 2 : 1;
#pragma unroll UNROLL
    for (int k = 0; k < H + 4; ++k) {
        int r = j0 - 2 + k;
        T h, qx, qy, zx, zy;
        T c_h, c_qx, c_qy;
        if constexpr (TMA_RING) {
            ring_arrive(k);
            const T *rowp = ring_row(k);
            h = rowp[FH * RR * NTX];
            qx = rowp[FQX * RR * NTX];
            qy = rowp[FQY * RR * NTX];
            zx = rowp[FZX * RR * NTX];
            zy = fp64 ? zx : rowp[FZY * RR * NTX];
            c_h = c_qx = c_qy = T(0);
            if (STAGE == 2 && un_ok(k)) {
                c_h = rowp[(FUN + 0) * RR * NTX];
                c_qx = rowp[(FUN + 1) * RR * NTX];
                c_qy = rowp[(FUN + 2) * RR * NTX];
            }
        } else {
            h = nh; qx = nqx; qy = nqy; zx = nzx; zy = nzy;
            if (k + 1 < H + 4) load(r + 1, nh, nqx, nqy, nzx, nzy);
            c_h = un_h; c_qx = un_qx; c_qy = un_qy;
        }
        T c_n2 = pn2, c_vi = pvi, c_ks = pks;
        prefetch(r - 1);
        Cell<T> rc = make_cell(h, qx, qy, zy, C.hdry);
        bool in_tile = r >= j0 && r < j0 + H && r < P.ny;     // uniform over the CTA
        if (in_tile) {
            s_st[t] = {rc.h, rc.u, rc.v, rc.rh};
            s_zx[t] = zx;
        }

        // ---- dry run: one CTA vote per row ----
        // With the input ring, every row is voted on: h = 0 in every column
        // of the CTA (and, in stage 2, U^n of the row updated now is +0).
        // After FAST consecutive such rows the iteration's results are known
        // exactly: rows r-4..r dry make every x part, y reconstruction and
        // y face of rows r-3..r-1 +0 (dry-dry faces, the cases above), so
        // row r-2 is quiet and its stage result is (+0, 0, 0) -- in stage 2,
        // with U^n = +0 and no rain or infiltration, also U^{n+1}; rows
        // r-6..r dry (stage 2) make U^{n+1} of rows r-4..r-2 +0, so the
        // fused wave speeds add nothing.  The pipeline registers already
        // hold those +0s; the iteration stores the zeros and shifts the
        // window (u = v = 1/h = 0 for dry cells, as make_cell gives).
        bool vote = false;
        if constexpr (DRY_SKIP && TMA_RING) {
            const bool rowdry = is0(rc.h) && (STAGE == 1 || (bits(c_h) | bits(c_qx) | bits(c_qy)) == 0);
            vote = cta_and<NTX>(rowdry);
            // every thread is past its reads of the block holding rows up to
            // r - 3 (the reload below reads rows r - 2 and r - 1): its slot
            // takes the block RD - 1 ahead
            if (t == 0 && k >= 2 && ((k - 2) & (RR - 1)) == 0) issue_block((k - 2) / RR + RD - 1);
            dryrun = vote ? dryrun + 1 : 0;
            constexpr int FAST = STAGE == 1 ? 5 : 7;
            if (dryrun >= FAST && (STAGE == 1 || (!rain && !P.infiltration))) {
                // The dry run: an inner loop whose only state is k and the
                // run length, so the registers of the general path stay where
                // they are; each row stores its zeros and votes on the next.
                T *const oh = STAGE == 1 ? F.h1 : F.h;
                T *const oqx = STAGE == 1 ? F.qx1 : F.qx;
                T *const oqy = STAGE == 1 ? F.qy1 : F.qy;
                const bool edge_col = gi < 2 || gi >= P.nx - 2;
                auto store_row = [&](int kk) {          // the zeros of the row updated at row kk
                    const int ro = j0 - 4 + kk;
                    if (kk >= 4 && ro < P.ny && out_col) {
                        if (edge_col || ro < 2 || ro >= P.ny - 2) {
                            store_cell<T>(P, oh, oqx, oqy, gi, ro, T(0), T(0), T(0));
                        } else {
                            const size_t o = pidx(P, gi, ro);
                            oh[o] = T(0);
                            oqx[o] = T(0);
                            oqy[o] = T(0);
                        }
                    }
                };
                auto row_dry = [&](int kk) {            // this thread's cells of row kk vote dry
                    const T *rowp = ring_row(kk);
                    bool rd = is0(rowp[FH * RR * NTX]);
                    if (STAGE == 2 && un_ok(kk))
                        rd = rd && (bits(rowp[(FUN + 0) * RR * NTX]) | bits(rowp[(FUN + 1) * RR * NTX]) |
                                    bits(rowp[(FUN + 2) * RR * NTX])) == 0;
                    return rd;
                };
                for (;;) {
                    store_row(k);
                    if (++k >= H + 4) break;
                    if ((k & (RR - 1)) == 0 && k + RR <= H + 4) {
                        // a whole ring block: one vote for its RR rows.  If
                        // all are dry, every row of it is fast (the run only
                        // grows) and no row of the block before is read
                        // again (a run can end no earlier than the next
                        // block), so that block's slot takes its successor
                        // now -- the one a row-by-row pass issues at row k + 2.
                        ring_arrive(k);
                        bool rd = true;
#pragma unroll
                        for (int i = 0; i < RR; ++i) rd = rd && row_dry(k + i);
                        if (cta_and<NTX>(rd)) {
                            if (t == 0) issue_block(k / RR + RD - 1);
                            dryrun += RR;
#pragma unroll
                            for (int i = 0; i < RR - 1; ++i) store_row(k + i);
                            k += RR - 1;                // the block's last row is stored above
                            continue;
                        }
                    }
                    ring_arrive(k);
                    vote = cta_and<NTX>(row_dry(k));
                    if (t == 0 && ((k - 2) & (RR - 1)) == 0) issue_block((k - 2) / RR + RD - 1);
                    dryrun = vote ? dryrun + 1 : 0;
                    if (dryrun < FAST) break;
                }
                if (k >= H + 4) break;
                // Row k ends the run and takes the general path: its inputs,
                // the window rows k-2 and k-1 (dry) read again from the ring,
                // the per-cell maps of row k-2, and its row published for the
                // x part.
                r = j0 - 2 + k;
                const T *rowp = ring_row(k);
                h = rowp[FH * RR * NTX];
                qx = rowp[FQX * RR * NTX];
                qy = rowp[FQY * RR * NTX];
                zx = rowp[FZX * RR * NTX];
                zy = fp64 ? zx : rowp[FZY * RR * NTX];
                c_h = c_qx = c_qy = T(0);
                if (STAGE == 2 && un_ok(k)) {
                    c_h = rowp[(FUN + 0) * RR * NTX];
                    c_qx = rowp[(FUN + 1) * RR * NTX];
                    c_qy = rowp[(FUN + 2) * RR * NTX];
                }
                const T *p2 = ring_row(k - 2), *p1 = ring_row(k - 1);
                ra = make_cell(p2[FH * RR * NTX], p2[FQX * RR * NTX], p2[FQY * RR * NTX],
                               fp64 ? p2[FZX * RR * NTX] : p2[FZY * RR * NTX], C.hdry);
                rb = make_cell(p1[FH * RR * NTX], p1[FQX * RR * NTX], p1[FQY * RR * NTX],
                               fp64 ? p1[FZX * RR * NTX] : p1[FZY * RR * NTX], C.hdry);
                prefetch(r - 2);
                c_n2 = pn2; c_vi = pvi; c_ks = pks;
                prefetch(r - 1);
                rc = make_cell(h, qx, qy, zy, C.hdry);
                in_tile = r >= j0 && r < j0 + H && r < P.ny;
                if (in_tile) {
                    s_st[t] = {rc.h, rc.u, rc.v, rc.rh};
                    s_zx[t] = zx;
                }
                cta_sync<NTX>();
            }
        }

        // ---- x part of row r (only rows this CTA updates) ----
        T a1 = T(0), a2 = T(0), a3 = T(0);
        if (in_tile) {
            // A row with h = 0 in every column of the CTA has zero x fluxes
            // and a zero Fc (h_- + h_+ = 0): its x differences are +0, the
            // value a1..a3 already hold, so the CTA skips the x part.  (With
            // the ring the vote above decides, conservatively: it also asks
            // for U^n = +0 in stage 2.)
            bool skip_x;
            if constexpr (DRY_SKIP && TMA_RING)
                skip_x = vote;
            else
                skip_x = DRY_SKIP ? cta_and<NTX>(is0(rc.h)) : (cta_sync<NTX>(), false);
            if (!skip_x) {
            Rec<T> q{};
            const bool rec = t >= 1 && t <= NTX - 2;
            V4<T> L{}, R{};
            if (rec) {
                L = s_st[t - 1];
                R = s_st[t + 1];
            }
            // A cell with h = 0 beside neighbours with h = 0 reconstructs
            // h_- = h_+ = 0 and u = v = 0 on both faces: both its faces are
            // dry on each side (their fluxes are +0 whatever the
            // reconstructed z), and its centred term is +0.  Such a thread
            // publishes the minus side (0, 0, 0, 0), which gives its west
            // neighbour's face the same zeros.
            const bool xdry = DRY_SKIP && is0(L.x) && is0(rc.h) && is0(R.x);
            T fcx = T(0);                 // centred x source term (+0 when skipped)
            if (rec && !xdry) {
                if constexpr (ORD1)
                    q = rec1<T>(rc.h, fp64 ? zx : T(0), rc.u, rc.v);
                else if constexpr (fp64)
                    q = muscl<T>(L.x, rc.h, R.x, s_zx[t - 1], zx, s_zx[t + 1],
                                 L.y, rc.u, R.y, L.z, rc.v, R.z, rc.rh, C.hdry);
                else
                    q = muscl<T>(L.x, rc.h, R.x, s_zx[t - 1], zx, T(0),
                                 L.y, rc.u, R.y, L.z, rc.v, R.z, rc.rh, C.hdry);
                fcx = hg * (q.hm + q.hp) * (q.zp - q.zm);
            }
            if (rec) s_m[t] = {q.hm, q.zm, q.unm, q.utm};
            cta_sync<NTX>();
            V4<T> fe{};
            if (t >= 1 && t <= NTX - 3) {
                // east face of a dry cell with a dry east neighbour: both
                // face depths are 0, every flux component +0
                if (!(DRY_SKIP && is0(rc.h) && is0(R.x))) {
                    V4<T> Rm = s_m[t + 1];
                    face_flux<T>(C.g, q.hp, q.zp, q.unp, q.utp, Rm.x, Rm.y, Rm.z, Rm.w, fp64 ? T(0) : zx,
                                 fe.x, fe.y, fe.z, fe.w);
                }
                s_f[t] = fe;
            }
            cta_sync<NTX>();
            if (out_col) {
                if (STAGE == 2 && P.check_cfl)
                    k2x = kmax(k2x, speed_key(mx(ab(q.unm) + sq(C.g * q.hm), ab(q.unp) + sq(C.g * q.hp))));
                V4<T> fw = s_f[t - 1];
                a1 = fe.x - fw.x;
                a2 = (fe.y - fw.z) + fcx;
                a3 = fe.w - fw.w;
                if (gi == 0 && P.bc[0] != SWOF_BC_WALL) outacc -= fw.x * cdy;
                if (gi == P.nx - 1 && P.bc[1] != SWOF_BC_WALL) outacc += fe.x * cdy;
            }
            }
        }

        // ---- y part: recon of row r-1, face between r-2 and r-1, update of r-2 ----
        if (k >= 2) {
            // Three dry cells down the column (h = 0 exactly): a dry cell's
            // reconstructed depths are 0 on both faces, so the face above it
            // and the face below it are dry-dry and their fluxes are exact
            // zeros whatever the reconstructed z; the centred term is 0 and
            // the speeds are 0.  The thread skips the reconstruction and the
            // face (no barrier involved; the result is the full path's).
            Rec<T> qb{};
            V4<T> gn{};
            T fcyb = T(0);                // centred y source term of row r-1 (+0 when skipped)
            const bool ydry = DRY_SKIP && is0(ra.h) && is0(rb.h) && is0(rc.h);
            if (!ydry) {
                if constexpr (ORD1)
                    qb = rec1<T>(rb.h, fp64 ? rb.zy : T(0), rb.v, rb.u);
                else if constexpr (fp64)
                    qb = muscl<T>(ra.h, rb.h, rc.h, ra.zy, rb.zy, rc.zy, ra.v, rb.v, rc.v, ra.u, rb.u, rc.u,
                                  rb.rh, C.hdry);
                else
                    qb = muscl<T>(ra.h, rb.h, rc.h, ra.zy, rb.zy, T(0), ra.v, rb.v, rc.v, ra.u, rb.u, rc.u,
                                  rb.rh, C.hdry);
                if (STAGE == 2 && P.check_cfl && out_col && r - 1 >= j0 && r - 1 < j0 + H && r - 1 < P.ny)
                    k2y = kmax(k2y, speed_key(mx(ab(qb.unm) + sq(C.g * qb.hm), ab(qb.unp) + sq(C.g * qb.hp))));
                if (k >= 3)
                    face_flux<T>(C.g, ypa.x, ypa.y, ypa.z, ypa.w, qb.hm, qb.zm, qb.unm, qb.utm,
                                 fp64 ? T(0) : ra.zy, gn.x, gn.y, gn.z, gn.w);
                fcyb = hg * (qb.hm + qb.hp) * (qb.zp - qb.zm);
            }
            const int ro = r - 2;                      // row updated now
            T fh = T(0), fu = T(0), fv = T(0), frh = T(0);
            if (k >= 4 && ro < P.ny && out_col) {
                // A cell at h = +0 whose x and y flux differences and centred
                // terms are all +0 ends the stage at (+0, 0, 0) -- what the
                // update below gives (+0 - dt/dx (+0) - dt/dy (+0), then
                // q := 0 below h_dry) -- so it skips the arithmetic; the test
                // is one OR of the bit patterns.
                const bool quiet = DRY_SKIP && (bits(ra.h) | bits(a1q[0]) | bits(a2q[0]) | bits(a3q[0]) |
                                                bits(gn.x) | bits(gs.x) | bits(gn.y) | bits(gs.z) | bits(fcya) |
                                                bits(gn.w) | bits(gs.w)) == 0;
                T hs = T(0), qxs = T(0), qys = T(0);
                if (!quiet) {
                T b1 = gn.x - gs.x;
                T b2 = (gn.y - gs.z) + fcya;
                T b3 = gn.w - gs.w;
                hs = ra.h - dtdx * a1q[0] - dtdy * b1;
                qxs = ra.qx - dtdx * a2q[0] - dtdy * b3;
                qys = ra.qy - dtdx * a3q[0] - dtdy * b2;
                }
                size_t o = pidx(P, gi, ro);
                if (quiet) {
                } else if (gt_pos(hs, C.hdry)) {
                    if (P.friction != SWOF_FRIC_NONE) {
                        // q / (1 + dt g C_f |u^s| / h*^p), p = 4/3 (Manning,
                        // Strickler) or 1 (Darcy-Weisbach, Chezy), Sec. 2.1, 3.2
                        T cf = c_n2;
                        T speed = sq(ra.u * ra.u + ra.v * ra.v);
                        T hinv;
                        if (P.friction <= SWOF_FRIC_STRICKLER) {
                            T y = icbrt(hs);
                            hinv = (y * y) * (y * y);
                        } else {
                            hinv = rcp(hs);
                        }
                        T den = T(1) + (dt * C.g * cf) * speed * hinv;
                        T rden = rcp(den);
                        qxs = qxs * rden;
                        qys = qys * rden;
                    }
                } else {
                    qxs = T(0);
                    qys = T(0);
                }
                if (ro == 0 && P.bc[2] != SWOF_BC_WALL) outacc -= gs.x * cdx;
                if (ro == P.ny - 1 && P.bc[3] != SWOF_BC_WALL) outacc += gn.x * cdx;
                if (STAGE == 1) {
                    store_cell<T>(P, F.h1, F.qx1, F.qy1, gi, ro, hs, qxs, qys);
                } else if (quiet && !rain && !P.infiltration && (bits(c_h) | bits(c_qx) | bits(c_qy)) == 0) {
                    // ... and with U^n = (+0, +0, +0), no rain and no
                    // infiltration U^{n+1} is (+0, +0, +0) (the Heun average
                    // of zeros; below h_dry)
                    store_cell<T>(P, F.h, F.qx, F.qy, gi, ro, T(0), T(0), T(0));
                } else {
                    // Heun average (U^n + U**)/2, then rain.  FP32 adds the
                    // step's rain to the Heun increment (U** - U^n)/2 before
                    // that meets U^n, so the depth is rounded once, and that
                    // rounding is stochastic (sr_add): the increment of a deep
                    // cell is of the order of its ulp, and rounded to nearest
                    // it would be lost or rounded up the same way every step.
                    T hn, qxn, qyn;
                    if constexpr (fp64) {
                        hn = T(0.5) * (c_h + hs);
                        qxn = T(0.5) * (c_qx + qxs);
                        qyn = T(0.5) * (c_qy + qys);
                        if (rain) hn = hn + rdt;
                    } else {
                        T dh = T(0.5) * (hs - c_h);
                        if (rain) dh = dh + rdt;
                        hn = sr_add(c_h, dh, (unsigned)(ro * P.nx + gi), sr_ts);
                        qxn = c_qx + T(0.5) * (qxs - c_qx);
                        qyn = c_qy + T(0.5) * (qys - c_qy);
                    }
                    if (P.infiltration) {
                        T vi = c_vi;
                        T ks = c_ks;
                        T d;
                        if (vi > T(0)) {
                            T ic = ks * (T(1) + ((C.psi + hn) * C.dtheta) / vi);
                            d = mn(hn, dt * ic);
                        } else {
                            d = hn;
                        }
                        hn = hn - d;
                        F.vinf[o] = vi + d;
                        infacc += d;
                    }
                    if (le_pos(hn, C.hdry)) {
                        qxn = T(0);
                        qyn = T(0);
                    }
                    store_cell<T>(P, F.h, F.qx, F.qy, gi, ro, hn, qxn, qyn);
                    fh = hn;
                    if (gt_pos(hn, C.hdry)) {
                        frh = rcp(hn);
                        fu = qxn * frh;
                        fv = qyn * frh;
                    }
                }
            }
            // wave speeds of U^{n+1} (Eq. (cfl)) for cells whose neighbours
            // this CTA owns; the tile-edge columns/rows are left to the ring
            // kernel of the next step
            if (STAGE == 2 && P.fuse_lambda && k >= 4) {       // uniform over the CTA
                V4<T> *buf = S.nw[k & 1];
                buf[t] = {fh, fu, fv, frh};
                // all three rows of U^{n+1} dry across the CTA: every speed is 0
                // (the same vote tells the tile flags whether the tile holds water)
                const bool alldry = DRY_SKIP ? cta_and<NTX>(is0(fh) && is0(y1h) && is0(y2h))
                                             : (cta_sync<NTX>(), false);
                anywet |= !alldry;
                if (!alldry && out_col && ro < P.ny) {
                    // a cell whose three cells along a direction hold h = 0 has
                    // face depths 0 and velocities 0: its speed is 0
                    if (xlam) {
                        V4<T> L = buf[t - 1], R = buf[t + 1];
                        if (!(DRY_SKIP && is0(L.x) && is0(fh) && is0(R.x)))
                            lx = kmax(lx, speed_key(cell_speed(L.x, fh, R.x, L.y, fu, R.y, frh, C.hdry, C.g)));
                    }
                    const int rr = ro - 1;
                    if (rr >= j0 + 1 && rr <= j0 + H - 2 && rr <= P.ny - 2 &&
                        !(DRY_SKIP && is0(y2h) && is0(y1h) && is0(fh)))
                        ly = kmax(ly, speed_key(cell_speed(y2h, y1h, fh, y2v, y1v, fv, y1rh, C.hdry, C.g)));
                }
                y2h = y1h;
                y2v = y1v;
                y1h = fh;
                y1v = fv;
                y1rh = frh;
            }
            // shift the y pipeline (a dry window's centred term is
            // hg (0 + 0)(0 - 0) = +0)
            ypa = {qb.hp, qb.zp, qb.unp, qb.utp};
            fcya = fcyb;
            gs = gn;
        }
        a1q[0] = a1q[1]; a2q[0] = a2q[1]; a3q[0] = a3q[1];
        a1q[1] = a1; a2q[1] = a2; a3q[1] = a3;
        ra = rb;
        rb = rc;
    }
    if constexpr (TMA_RING) {
        if (!ring_ok) {
            // a ring wait ran out: report it, and give the copies still in
            // flight (bounded) time to land before the CTA's shared memory
            // is released
            atomicExch(const_cast<int *>(&ctl->status), SWOF_ETIMEOUT);
            if (t == 0)
                for (int b = nblk - RD > 0 ? nblk - RD : 0; b < nblk; ++b)
                    ring_wait(tc05::smem_u32(&S.bar[b % RD]), (uint32_t)((b / RD) & 1));
        }
    }
    }

    // FP64 budget slots, fixed order (one Euler stage at first order, else
    // each Heun stage counts half)
    // (a tile left alone adds nothing anywhere: its sums and maxima are 0)
    const bool edge = (bx == 0 && P.bc[0] != SWOF_BC_WALL) || (bx == gdx - 1 && P.bc[1] != SWOF_BC_WALL) ||
                      (by == 0 && P.bc[2] != SWOF_BC_WALL) || (by == gdy - 1 && P.bc[3] != SWOF_BC_WALL);
    if (edge && !P.no_budget && !dead) {
        double s = block_sum_t(outacc, s_red);
        if (t == 0) F.outflow_slots[blk] += (ORD1 ? 1.0 : 0.5) * ctl->dt * s;
    }
    if (STAGE == 2 && F.tile_act && t == 0 && !dead) F.tile_act[blk] = (unsigned char)anywet;
    if (STAGE == 2 && P.infiltration && !P.no_budget && !dead) {
        double s = block_sum_t(infacc, s_red);
        if (t == 0) F.infil_slots[blk] += s;
    }
    if (STAGE == 2 && P.fuse_lambda && !dead) {
        lx = block_max(lx, S.redk[0]);
        ly = block_max(ly, S.redk[1]);
        if (t == 0) {      // (a zero maximum changes nothing)
            if (lx) atomicMax(&F.ctl->lam_bits[0], key64(lx));
            if (ly) atomicMax(&F.ctl->lam_bits[1], key64(ly));
        }
    }
    if (STAGE == 2 && P.check_cfl) {
        if (!dead) {
            k2x = block_max(k2x, S.redk[0]);
            k2y = block_max(k2y, S.redk[1]);
        }
        if (t == 0) {
            DevCtl *c = F.ctl;
            atomicMax(&c->lam2_bits[0], key64(k2x));
            atomicMax(&c->lam2_bits[1], key64(k2y));
            __threadfence();
            unsigned int nb = (unsigned int)(gdx * gdy);
            if (atomicAdd(&c->done2, 1u) == nb - 1) {
                __threadfence();
                double lx = __longlong_as_double((long long)atomicAdd(&c->lam2_bits[0], 0ull));
                double ly = __longlong_as_double((long long)atomicAdd(&c->lam2_bits[1], 0ull));
                c->lam2_bits[0] = 0ull;
                c->lam2_bits[1] = 0ull;
                c->done2 = 0u;
                if (c->dt * (lx / P.dx + ly / P.dy) > P.cfl) c->cfl_viol++;
            }
        }
    }
}

// (No minimum-blocks hint: capping registers that way made the compiler
// route work through the FP64 pipe, which on GB300 costs more than the
// occupancy it buys.)  The input ring lives in dynamic shared memory
// (ring_bytes<T, STAGE, NTX>(), opted in per device by configure_t), the tensor
// maps of the fields in parameter space.
// The same stage with the one-row register prefetch instead of the ring
// (and so without the dry fast path): on grids wet almost everywhere every
// row takes the full path, and this form keeps more CTAs per SM (no ring in
// shared memory).  The tile-shape tuner times both forms.
template <typename T, int STAGE, int NTX, int H, bool ORD1 = false>
__global__ void __launch_bounds__(NTX) k_sweep_reg(Params P, Fields<T> F)
{
    __shared__ SweepSmem<T, NTX> S;
    sweep_tile<T, STAGE, NTX, H, true, ORD1, false>(P, F, blockIdx.x, blockIdx.y, gridDim.x, gridDim.y, S);
}

template <typename T, int STAGE, int NTX, int H, bool ORD1 = false>
__global__ void __launch_bounds__(NTX) k_sweep(Params P, Fields<T> F, const __grid_constant__ SweepMaps M)
{
    __shared__ SweepSmem<T, NTX> S;
    extern __shared__ __align__(128) unsigned char sweep_dyn[];
    T *ring = reinterpret_cast<T *>(sweep_dyn);
    sweep_tile<T, STAGE, NTX, H, true, ORD1, true>(P, F, blockIdx.x, blockIdx.y, gridDim.x, gridDim.y, S, ring, &M);
}

SWOF_KERNELS_END

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
// Every input cell is read from HBM once (next row prefetched), every output
// written once.  The per-cell arithmetic is exactly the one of the oracle
// (same functions, same operation order), so the FP64 instantiation stays
// bit-identical to it; work whose result is known exactly is skipped: the x
// part of a row dry across the CTA, the y part of a column window of three
// dry cells, and (FP64) the update of a dry cell whose fluxes are all +0.
#pragma once

namespace swof {

template <typename T>
struct Cell {
    T h, u, v, rh, qx, qy, zy;
};

template <typename T>
__device__ __forceinline__ Cell<T> make_cell(T h, T qx, T qy, T zy, T hdry)
{
    Cell<T> c = {h, T(0), T(0), T(0), qx, qy, zy};
    if (h > hdry) {
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

// x == 0 of either sign; FP64 on the bit pattern, off GB300's narrow FP64
// pipe (same answer as the comparison, NaN included).
__device__ __forceinline__ bool is0(double x) { return (__double_as_longlong(x) << 1) == 0; }
__device__ __forceinline__ bool is0(float x) { return x == 0.0f; }
__device__ __forceinline__ unsigned long long bits(double x) { return (unsigned long long)__double_as_longlong(x); }

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
};

// One stage over the tile (bx, by) of a (gdx x gdy) tiling; the kernel
// below maps it to its block index, the ensemble kernel to a queue item.
// DRY_SKIP: let a CTA skip the x part of a row (and the wave speeds of three
// rows) that is dry across its columns -- exact, and a large saving on
// mostly dry grids; grids that are wet everywhere (the ensemble's rain
// scenarios) run without the vote.
// ORD1: the first-order stage (Sec. 3.3): face values = cell values.
// With F.tile_act set (dry-tile skipping), a tile whose 3x3 tile
// neighbourhood held no water after the last step, with no rain and no
// imposed edge, is left alone: every flux of the step is exactly zero there
// and U^{n+1} = U^n (stage 2 works in place); stage 1 writes its U* = 0 once
// when the tile turns dry, for the neighbours' halos.
template <typename T, int STAGE, int NTX, int H, bool DRY_SKIP = true, bool ORD1 = false>
__device__ __forceinline__ void sweep_tile(const Params &P, const Fields<T> &F, int bx, int by, int gdx, int gdy,
                                           SweepSmem<T, NTX> &S)
{
    constexpr bool fp64 = std::is_same<T, double>::value;
    constexpr int W = NTX - 4;
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
    // iteration ahead: U^n (stage 2), n^2 map, V_inf and K_s
    T un_h = T(0), un_qx = T(0), un_qy = T(0), pn2 = C.cf, pvi = T(0), pks = C.ks;
    const bool want_prefetch = STAGE == 2 || F.cfmap != nullptr;
    auto prefetch = [&](int ro) {
        if (!want_prefetch || !(out_col && ro >= j0 && ro < j0 + H && ro < P.ny)) return;
        size_t o = pidx(P, gi, ro);
        if (STAGE == 2) {
            un_h = F.h[o];
            un_qx = F.qx[o];
            un_qy = F.qy[o];
            if (P.infiltration) {
                pvi = F.vinf[o];
                if (F.ksmap) pks = F.ksmap[o];
            }
        }
        if (F.cfmap) pn2 = F.cfmap[o];
    };

    bool anywet = false;                // a row of U^{n+1} of this tile holds water (stage 2, uniform)
    if (!dead) {
    T nh, nqx, nqy, nzx, nzy;
    load(j0 - 2, nh, nqx, nqy, nzx, nzy);
    // two rows per trip in the stage kernels: the register window rotates
    // by renaming instead of moves (measured ~1.5 % per stage; three rows
    // per trip raised register use and was slower).  The ensemble's
    // persistent kernel (no dry vote) keeps its own register budget.
    constexpr int UNROLL = DRY_SKIP ? 2 : 1;
#pragma unroll UNROLL
    for (int k = 0; k < H + 4; ++k) {
        const int r = j0 - 2 + k;
        T h = nh, qx = nqx, qy = nqy, zx = nzx, zy = nzy;
        if (k + 1 < H + 4) load(r + 1, nh, nqx, nqy, nzx, nzy);
        T c_h = un_h, c_qx = un_qx, c_qy = un_qy, c_n2 = pn2, c_vi = pvi, c_ks = pks;
        prefetch(r - 1);
        Cell<T> rc = make_cell(h, qx, qy, zy, C.hdry);

        // ---- x part of row r (only rows this CTA updates) ----
        T a1 = T(0), a2 = T(0), a3 = T(0);
        if (r >= j0 && r < j0 + H && r < P.ny) {     // uniform over the CTA
            s_st[t] = {rc.h, rc.u, rc.v, rc.rh};
            s_zx[t] = zx;
            // A row with h = 0 in every column of the CTA has zero x fluxes
            // and a zero Fc (h_- + h_+ = 0): its x differences are +0, the
            // value a1..a3 already hold, so the CTA skips the x part.
            if (!(DRY_SKIP ? cta_and<NTX>(is0(rc.h)) : (cta_sync<NTX>(), 0))) {
            Rec<T> q{};
            const bool rec = t >= 1 && t <= NTX - 2;
            if (rec) {
                V4<T> L = s_st[t - 1], R = s_st[t + 1];
                if constexpr (ORD1)
                    q = rec1<T>(rc.h, fp64 ? zx : T(0), rc.u, rc.v);
                else if constexpr (fp64)
                    q = muscl<T>(L.x, rc.h, R.x, s_zx[t - 1], zx, s_zx[t + 1],
                                 L.y, rc.u, R.y, L.z, rc.v, R.z, rc.rh, C.hdry);
                else
                    q = muscl<T>(L.x, rc.h, R.x, s_zx[t - 1], zx, T(0),
                                 L.y, rc.u, R.y, L.z, rc.v, R.z, rc.rh, C.hdry);
                s_m[t] = {q.hm, q.zm, q.unm, q.utm};
            }
            cta_sync<NTX>();
            V4<T> fe{};
            if (t >= 1 && t <= NTX - 3) {
                V4<T> R = s_m[t + 1];
                face_flux<T>(C.g, q.hp, q.zp, q.unp, q.utp, R.x, R.y, R.z, R.w, fp64 ? T(0) : zx,
                             fe.x, fe.y, fe.z, fe.w);
                s_f[t] = fe;
            }
            cta_sync<NTX>();
            if (out_col) {
                if (STAGE == 2 && P.check_cfl)
                    k2x = kmax(k2x, speed_key(mx(ab(q.unm) + sq(C.g * q.hm), ab(q.unp) + sq(C.g * q.hp))));
                V4<T> fw = s_f[t - 1];
                T fcx = hg * (q.hm + q.hp) * (q.zp - q.zm);
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
            }
            const int ro = r - 2;                      // row updated now
            T fh = T(0), fu = T(0), fv = T(0), frh = T(0);
            if (k >= 4 && ro < P.ny && out_col) {
                // FP64: a cell at h = +0 whose x and y flux differences and
                // centred terms are all +0 ends the stage at (+0, 0, 0) -- what
                // the update below gives (+0 - dt/dx (+0) - dt/dy (+0), then
                // q := 0 below h_dry) -- so it skips the FP64 arithmetic; the
                // test is one OR of the bit patterns.
                bool quiet = false;
                if constexpr (fp64)
                    quiet = DRY_SKIP && (bits(ra.h) | bits(a1q[0]) | bits(a2q[0]) | bits(a3q[0]) | bits(gn.x) |
                                         bits(gs.x) | bits(gn.y) | bits(gs.z) | bits(fcya) | bits(gn.w) |
                                         bits(gs.w)) == 0ull;
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
                } else if (hs > C.hdry) {
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
                } else if (quiet && !rain && !P.infiltration && (bits(c_h) | bits(c_qx) | bits(c_qy)) == 0ull) {
                    // ... and with U^n = (+0, +0, +0), no rain and no
                    // infiltration U^{n+1} is (+0, +0, +0) (the Heun average
                    // of zeros; below h_dry)
                    store_cell<T>(P, F.h, F.qx, F.qy, gi, ro, T(0), T(0), T(0));
                } else {
                    T hn = T(0.5) * (c_h + hs);
                    T qxn = T(0.5) * (c_qx + qxs);
                    T qyn = T(0.5) * (c_qy + qys);
                    if (rain) hn = hn + rdt;
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
                    if (hn <= C.hdry) {
                        qxn = T(0);
                        qyn = T(0);
                    }
                    store_cell<T>(P, F.h, F.qx, F.qy, gi, ro, hn, qxn, qyn);
                    fh = hn;
                    if (hn > C.hdry) {
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
                    if (xlam) {
                        V4<T> L = buf[t - 1], R = buf[t + 1];
                        lx = kmax(lx, speed_key(cell_speed(L.x, fh, R.x, L.y, fu, R.y, frh, C.hdry, C.g)));
                    }
                    const int rr = ro - 1;
                    if (rr >= j0 + 1 && rr <= j0 + H - 2 && rr <= P.ny - 2)
                        ly = kmax(ly, speed_key(cell_speed(y2h, y1h, fh, y2v, y1v, fv, y1rh, C.hdry, C.g)));
                }
                y2h = y1h;
                y2v = y1v;
                y1h = fh;
                y1v = fv;
                y1rh = frh;
            }
            // shift the y pipeline
            ypa = {qb.hp, qb.zp, qb.unp, qb.utp};
            fcya = hg * (qb.hm + qb.hp) * (qb.zp - qb.zm);
            gs = gn;
        }
        a1q[0] = a1q[1]; a2q[0] = a2q[1]; a3q[0] = a3q[1];
        a1q[1] = a1; a2q[1] = a2; a3q[1] = a3;
        ra = rb;
        rb = rc;
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
// occupancy it buys.)
template <typename T, int STAGE, int NTX, int H, bool ORD1 = false>
__global__ void __launch_bounds__(NTX) k_sweep(Params P, Fields<T> F)
{
    __shared__ SweepSmem<T, NTX> S;
    sweep_tile<T, STAGE, NTX, H, true, ORD1>(P, F, blockIdx.x, blockIdx.y, gridDim.x, gridDim.y, S);
}

}  // namespace swof

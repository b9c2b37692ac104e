// mrlt_stage.cuh -- the stage kernels of the MR/MRLT time evolution: face
// fluxes from the exposures of Secs. 4.1-4.3, the compact RK update of Sec. 3
// and the flux-register epilogue.
// k_stage_tile (d = 1, 2, 3) works on one tile of one level per CTA: the
// halo is staged in shared memory and every face flux is computed once.  It is
// instantiated for R = double and, for the mixed-precision mode, R = float:
// reconstruction and numerical flux in R; the stored state, the right-hand
// side, the RK update and the flux registers stay in double.
#pragma once
#include "mrlt_impl.cuh"

namespace mrlt {

// Compact RK update of one leaf from its right-hand side f (Sec. 3):
//   s = 1: q*  = q^n + dt_l f
//   s = 2: RK2 q^{n+1} = q^n/2 + q*/2 + dt_l f/2 ; RK3 q** = 3q^n/4 + q*/4 + dt_l f/4
//   s = 3: q^{n+1} = q^n/3 + 2q**/3 + 2 dt_l f/3
// qs is the leaf's own value at stage s (q^n, q*, q** for s = 1, 2, 3: its
// exposure, already staged in shared memory) and q0 its q^n (s >= 2).
template <int M>
__device__ __forceinline__ void rk_update(const Grid& g, int u, long long id, int s, double dtl, const double* f,
                                          const double* q0, const double* qs)
{
    const long long N = g.N[u];
    double* q1 = fbase_w(g, F_Q1, u) + id;
    double* q2 = fbase_w(g, F_Q2, u) + id;
    double* qe = fbase_w(g, F_QE, u) + id;
#pragma unroll
    for (int v = 0; v < M; ++v) {
        const double kk = dtl * f[v];
        if (s == 1) {
            q1[v * N] = qs[v] + kk;
        } else if (s == 2) {
            if (g.rk == 2) qe[v * N] = 0.5 * q0[v] + 0.5 * qs[v] + 0.5 * kk;
            else q2[v * N] = 0.75 * q0[v] + 0.25 * qs[v] + 0.25 * kk;
        } else {
            qe[v * N] = (1.0 / 3.0) * q0[v] + (2.0 / 3.0) * qs[v] + (2.0 / 3.0) * kk;
        }
    }
}

// flux registers (conservation across levels): dt_l b_s F at coarse-fine faces
template <int M>
__device__ __forceinline__ void reg_add(const Grid& g, int u, long long id, int fi, int kind, double bw,
                                        const double* F)
{
    if (kind != K_FINER && kind != K_COARSER) return;
    const long long N = g.N[u];
    double* R = (kind == K_FINER ? g.rc : g.rf) + g.off[u] * g.nf * g.m + id;
#pragma unroll
    for (int v = 0; v < M; ++v) R[(fi * M + v) * N] += bw * F[v];
}

// Tile shapes of the tiled stage kernel: a CTA of THREADS threads owns
// TX x TY x TZ cells of one level (the same shapes index the per-level
// active-tile lists); THREADS may exceed the cell count, so that the list,
// exposure and face phases spread over more threads.
template <int D> struct Tile;
template <> struct Tile<1> { static constexpr int TX = kTile1X, TY = 1, TZ = 1, THREADS = kTileThreads1; };
template <> struct Tile<2> { static constexpr int TX = kTile2X, TY = kTile2Y, TZ = 1, THREADS = kTileThreads2; };
template <> struct Tile<3> { static constexpr int TX = kTile3X, TY = kTile3Y, TZ = kTile3Z, THREADS = kTileThreads3; };

// Block (tile + 2-cell ring) and face counts of one tile; the three large
// shared arrays (conservative values, reconstruction variables, face fluxes)
// live in dynamic shared memory, SMEM bytes.
template <int EQ, int D, class R>
struct TileShape {
    static constexpr int M = EQ == 2 ? D + 2 : 1;
    static constexpr int TX = Tile<D>::TX, TY = Tile<D>::TY, TZ = Tile<D>::TZ, H = 2;
    static constexpr int NC = TX * TY * TZ, NT = Tile<D>::THREADS; // cells, threads
    static_assert(NT % 32 == 0 && NT >= NC, "whole warps, at least one thread per cell");
    static constexpr int BX = TX + 2 * H, BY = D > 1 ? TY + 2 * H : 1, BZ = D > 2 ? TZ + 2 * H : 1;
    static constexpr int NB = BX * BY * BZ;
    static constexpr int NFX = (TX + 1) * TY * TZ;
    static constexpr int NFY = D > 1 ? TX * (TY + 1) * TZ : 0;
    static constexpr int NFZ = D > 2 ? TX * TY * (TZ + 1) : 0;
    static constexpr int NF = NFX + NFY + NFZ;
    static constexpr size_t SMEM = sizeof(double) * M * NB + sizeof(R) * M * NB + sizeof(R) * M * NF;
};

// Append, in thread order, `item` to list A where `ta` holds and to list B
// where `tb` holds, with one barrier per call.  The per-warp counts alternate
// between two halves of sWarp (2 x 2 x NT/32 ints, selected by `par`): a call
// may overwrite a half only after every thread has passed the barrier of the
// call in between, hence after every thread has read that half.  The caller
// issues a __syncthreads() before reading the lists.
template <int NT>
__device__ __forceinline__ void block_append2(bool ta, bool tb, int item, short* la, short* lb, int& na,
                                              int& nb, int* sWarp, int& par)
{
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned ba = __ballot_sync(0xffffffffu, ta);
    const unsigned bb = __ballot_sync(0xffffffffu, tb);
    int* w = sWarp + par * 2 * NW;
    if (lane == 0) {
        w[warp] = __popc(ba);
        w[NW + warp] = __popc(bb);
    }
    __syncthreads();
    int pa = 0, pb = 0, totA = 0, totB = 0;
#pragma unroll
    for (int i = 0; i < NW; ++i) {
        const int ca = w[i], cb = w[NW + i];
        pa += i < warp ? ca : 0;
        pb += i < warp ? cb : 0;
        totA += ca;
        totB += cb;
    }
    const unsigned below = (1u << lane) - 1u;
    if (ta) la[na + pa + __popc(ba & below)] = (short)item;
    if (tb) lb[nb + pb + __popc(bb & below)] = (short)item;
    na += totA;
    nb += totB;
    par ^= 1;
}

// Tiled stage (d = 1, 2, 3).  The CTA
//  1. reads the status of its tile and a 2-cell ring; tiles without leaves exit;
//  2. lists the cells some leaf of the tile reads -- its radius-2 cross stencil,
//     plus the 3^d block of a leaf facing an internal node -- and stages their
//     exposures (Secs. 4.1-4.3) and reconstruction variables in shared memory,
//     stored nodes first, then virtual cells and ghosts;
//  3. lists the faces touching a tile leaf and computes each once: plain faces
//     on level u from the shared cells; faces of a leaf against an internal node
//     as the mean of 2^{d-1} sub-face fluxes on level u+1 (Sec. 2), one thread
//     per sub-face (the 2^{d-1} threads of a face are adjacent lanes), the
//     leaf's virtual children predicted (Eq. 4) from its shared 3^d block and
//     the finer side read from level u+1;
//  4. applies the compact RK update and the register epilogue to its leaves.
// Work lists keep every warp on one kind of work.
template <int EQ, int D, class R>
__global__ void __launch_bounds__(Tile<D>::THREADS)
k_stage_tile(Grid g, int lo, int hi, int s, int lmin, double bstage, int reg)
{
    pdl_enter();
    const double dt = *g.dtp; // fine step of the macro step
    using S = TileShape<EQ, D, R>;
    constexpr int M = S::M, TX = S::TX, TY = S::TY, TZ = S::TZ, NT = S::NT, H = S::H;
    constexpr int BX = S::BX, BY = S::BY, NB = S::NB;
    constexpr int NFX = S::NFX, NFY = S::NFY, NF = S::NF;
    constexpr int NTS = 1 << (D - 1); // sub-faces per face
    constexpr int NL = NB > NF ? NB : NF;
    constexpr int OUT = 3;            // status code of a cell past a wall
    constexpr int SY = BX, SZ = BX * BY; // block strides in y and z
    extern __shared__ __align__(16) unsigned char smem[];
    double (*sW)[NB] = reinterpret_cast<double (*)[NB]>(smem);
    R (*sP)[NB] = reinterpret_cast<R (*)[NB]>(smem + sizeof(double) * M * NB);
    // x faces [0, NFX), y faces [NFX, NFX + NFY), z faces [NFX + NFY, NF)
    R (*sF)[NF] = reinterpret_cast<R (*)[NF]>(smem + (sizeof(double) + sizeof(R)) * M * NB);
    __shared__ uint8_t sSt[NB];
    __shared__ short sList[NL], sList2[NL];
    __shared__ int sWarp[4 * (NT / 32)];

    // The CTA walks the active tiles (tiles holding a leaf) of levels lo..hi,
    // in level order; one launch may cover several independent levels.
    __shared__ int sBase[LMAX + 2];
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int l = lo; l <= hi; ++l) {
            sBase[l - lo] = acc;
            acc += g.counts[2 * (LMAX + 1) + l];
        }
        sBase[hi - lo + 1] = acc;
    }
    __syncthreads();
    const int ntask = sBase[hi - lo + 1];
    for (int task = blockIdx.x; task < ntask; task += gridDim.x) {
    int li = 0;
    while (task >= sBase[li + 1]) ++li;
    const int u = lo + li;
    const int tile = g.tlist[g.toff[u] + task - sBase[li]];
    const double dtl = g.gts ? dt : ldexp(dt, g.L - u); // Eq. 13 step of level u
    const double bw = dtl * bstage; // register weight dt_l b_s
    const int n = g.n[u];
    const int ntx = (n + TX - 1) / TX, nty = (n + TY - 1) / TY;
    const int ox = (tile % ntx) * TX;
    const int oy = D > 1 ? ((tile / ntx) % nty) * TY : 0;
    const int oz = D > 2 ? (tile / (ntx * nty)) * TZ : 0;
    const int tid = threadIdx.x;
    const Ctx x{u, s, lmin};
    const bool finer = u < g.L; // internal nodes of level u have children

    // is block cell (bx, by, bz) a leaf of this tile?
    auto tile_leaf = [&](int bx, int by, int bz) -> bool {
        if (bx < H || bx >= H + TX || ox + bx - H >= n) return false;
        if (D > 1 && (by < H || by >= H + TY || oy + by - H >= n)) return false;
        if (D > 2 && (bz < H || bz >= H + TZ || oz + bz - H >= n)) return false;
        return sSt[bz * SZ + by * SY + bx] == 1;
    };
    // a tile leaf with an internal node across one of its faces
    auto leaf_li = [&](int bx, int by, int bz) -> bool {
        if (!finer || !tile_leaf(bx, by, bz)) return false;
        const int b = bz * SZ + by * SY + bx;
        bool li = sSt[b - 1] == 2 || sSt[b + 1] == 2;
        if (D > 1) li = li || sSt[b - SY] == 2 || sSt[b + SY] == 2;
        if (D > 2) li = li || sSt[b - SZ] == 2 || sSt[b + SZ] == 2;
        return li;
    };
    auto needed = [&](int b) -> bool {
        const int bx = b % BX, by = (b / BX) % BY, bz = b / SZ;
        bool need = false;
#pragma unroll
        for (int d = -2; d <= 2; ++d) {
            need = need || tile_leaf(bx + d, by, bz);
            if (D > 1) need = need || tile_leaf(bx, by + d, bz);
            if (D > 2) need = need || tile_leaf(bx, by, bz + d);
        }
#pragma unroll
        for (int dz = (D > 2 ? -1 : 0); dz <= (D > 2 ? 1 : 0); ++dz)
#pragma unroll
            for (int dy = (D > 1 ? -1 : 0); dy <= (D > 1 ? 1 : 0); ++dy)
#pragma unroll
                for (int dx = -1; dx <= 1; ++dx) need = need || leaf_li(bx + dx, by + dy, bz + dz);
        return need;
    };
    // geometry of face f: the cells on its two sides and the direction
    auto face = [&](int f, int& k, int& lo, int& hi, bool& leafLo, bool& leafHi) {
        if (f < NFX) {
            const int i = f % (TX + 1), r = f / (TX + 1), j = r % TY, kz = r / TY;
            const int by = D > 1 ? H + j : 0, bz = D > 2 ? H + kz : 0;
            k = 0;
            lo = bz * SZ + by * SY + H + i - 1;
            hi = lo + 1;
            leafLo = tile_leaf(H + i - 1, by, bz);
            leafHi = tile_leaf(H + i, by, bz);
        } else if (D < 3 || f < NFX + NFY) {
            const int ff = f - NFX, i = ff % TX, r = ff / TX, j = r % (TY + 1), kz = r / (TY + 1);
            const int bz = D > 2 ? H + kz : 0;
            k = 1;
            lo = bz * SZ + (H + j - 1) * SY + H + i;
            hi = lo + SY;
            leafLo = tile_leaf(H + i, H + j - 1, bz);
            leafHi = tile_leaf(H + i, H + j, bz);
        } else {
            const int ff = f - NFX - NFY, i = ff % TX, r = ff / TX, j = r % TY, kz = r / TY;
            k = 2;
            lo = (H + kz - 1) * SZ + (H + j) * SY + H + i;
            hi = lo + SZ;
            leafLo = tile_leaf(H + i, H + j, H + kz - 1);
            leafHi = tile_leaf(H + i, H + j, H + kz);
        }
    };

    // 1. status of the tile and its ring
    for (int b = tid; b < NB; b += NT) {
        const int bx = b % BX, by = (b / BX) % BY, bz = b / SZ;
        int qx, qy = 0, qz = 0;
        const bool inb = in_box(g, u, 0, ox + bx - H, &qx) && (D < 2 || in_box(g, u, 1, oy + by - H, &qy)) &&
                         (D < 3 || in_box(g, u, 2, oz + bz - H, &qz));
        sSt[b] = inb ? status(g, u, cell_id(g, u, qx, qy, qz)) : OUT;
    }
    __syncthreads();
    const int nleaf = __syncthreads_count(
        tid < S::NC && tile_leaf(H + tid % TX, D > 1 ? H + (tid / TX) % TY : 0, D > 2 ? H + tid / (TX * TY) : 0));
    if (nleaf == 0) continue; // uniform across the CTA
    if (tid == 0) {
        if (s == 1) atomicAdd(g.updates, (unsigned long long)nleaf);
        atomicAdd(&g.work[u * 4 + s], (unsigned long long)nleaf);
    }

    // 2. exposures of the needed cells: stored nodes (list 1), then virtual
    //    cells and ghosts (list 2)
    int nst = 0, nvc = 0, par = 0;
    for (int b0 = 0; b0 < NB; b0 += NT) {
        const int b = b0 + tid;
        const bool nd = b < NB && needed(b);
        const bool stored = nd && (sSt[b] == 1 || sSt[b] == 2);
        block_append2<NT>(stored, nd && !stored, b, sList, sList2, nst, nvc, sWarp, par);
    }
    __syncthreads();
    for (int t = tid; t < nst + nvc; t += NT) {
        const int b = t < nst ? sList[t] : sList2[t - nst];
        const int bx = b % BX, by = (b / BX) % BY, bz = b / SZ;
        double W[M];
        R P[M];
        if (t < nst) {
            int qx, qy = 0, qz = 0;
            in_box(g, u, 0, ox + bx - H, &qx);
            if (D > 1) in_box(g, u, 1, oy + by - H, &qy);
            if (D > 2) in_box(g, u, 2, oz + bz - H, &qz);
            expose<M>(g, x, u, cell_id(g, u, qx, qy, qz), sSt[b], W);
        } else {
            const int p[3] = {ox + bx - H, D > 1 ? oy + by - H : 0, D > 2 ? oz + bz - H : 0};
            value_at<D, M>(g, x, u, p, W);
        }
        recon_vars<EQ, D, M, R>(g, W, P);
#pragma unroll
        for (int v = 0; v < M; ++v) {
            sW[v][b] = W[v];
            sP[v][b] = P[v];
        }
    }
    __syncthreads();

    // 3. the faces touching a tile leaf, one pass: faces of a leaf against an
    //    internal node (list 1, 2^{d-1} sub-face tasks each, in adjacent
    //    lanes), then plain faces on level u (list 2), one thread per face
    int nsb = 0, nfl = 0;
    for (int f0 = 0; f0 < NF; f0 += NT) {
        const int f = f0 + tid;
        bool sub = false, plain = false;
        if (f < NF) {
            int k, lo, hi;
            bool lL, lH;
            face(f, k, lo, hi, lL, lH);
            sub = finer && ((lL && sSt[hi] == 2) || (lH && sSt[lo] == 2));
            plain = (lL || lH) && !sub;
        }
        block_append2<NT>(sub, plain, f, sList, sList2, nsb, nfl, sWarp, par);
    }
    __syncthreads();
    const int nsub = nsb * NTS; // sub-face tasks come first; NTS divides 32
    for (int base = 0; base < nsub + nfl; base += NT) {
        const int task = base + tid;
        const bool isSub = task < nsub, act = task < nsub + nfl;
        const int f = isSub ? sList[task / NTS] : (act ? sList2[task - nsub] : 0);
        const int t = isSub ? task % NTS : 0;
        R F[M];
#pragma unroll
        for (int v = 0; v < M; ++v) F[v] = R(0);
        if (act) {
            int k, lo, hi;
            bool lL, lH;
            face(f, k, lo, hi, lL, lH);
            if (!isSub) {
                const int stride = k == 0 ? 1 : (k == 1 ? SY : SZ);
                flux_recon<EQ, D, M, R>(g, k, g.dx[u][k], [&](int c, int v) { return sP[v][lo + (c - 1) * stride]; },
                                        F);
            } else {
                const bool leafIsLo = lL && sSt[hi] == 2;
                const int bl = leafIsLo ? lo : hi, side = leafIsLo ? 1 : -1;
                const int bx = bl % BX, by = (bl / BX) % BY, bz = bl / SZ;
                const int c[3] = {ox + bx - H, D > 1 ? oy + by - H : 0, D > 2 ? oz + bz - H : 0};
                // tangential directions of the face, in increasing order; sub-face
                // t takes child offset (t & 1) along the first, (t >> 1) along the second
                const int j1 = k == 0 ? 1 : 0, j2 = k == 2 ? 1 : 2;
                R P4[4][M];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    // stencil cell i on level u+1; the leaf's own children are virtual
                    int p[3] = {0, 0, 0};
                    p[k] = 2 * c[k] + (side > 0 ? i : i - 2);
                    if (D > 1) p[j1] = 2 * c[j1] + (t & 1);
                    if (D > 2) p[j2] = 2 * c[j2] + (t >> 1);
                    const bool own = side > 0 ? i < 2 : i >= 2;
                    double W[M];
                    if (own) {
                        const int ax = p[0] & 1, ay = p[1] & 1, az = p[2] & 1;
#pragma unroll
                        for (int v = 0; v < M; ++v) W[v] = 0.0;
#pragma unroll
                        for (int dz = (D > 2 ? -1 : 0); dz <= (D > 2 ? 1 : 0); ++dz)
#pragma unroll
                            for (int dy = (D > 1 ? -1 : 0); dy <= (D > 1 ? 1 : 0); ++dy)
#pragma unroll
                                for (int dx = -1; dx <= 1; ++dx) {
                                    const double w = ((D > 2 ? pw(az, dz) : 1.0) * (D > 1 ? pw(ay, dy) : 1.0)) *
                                                     pw(ax, dx);
                                    const int bs = bl + dz * SZ + dy * SY + dx;
#pragma unroll
                                    for (int v = 0; v < M; ++v) W[v] += w * sW[v][bs];
                                }
                    } else {
                        value_at<D, M>(g, x, u + 1, p, W);
                    }
                    recon_vars<EQ, D, M, R>(g, W, P4[i]);
                }
                flux_recon<EQ, D, M, R>(g, k, g.dx[u + 1][k], [&](int cc, int v) { return P4[cc][v]; }, F);
            }
        }
        // mean of the sub-face fluxes of a face (every lane takes part in the
        // shuffles; plain-face lanes keep their own flux)
        if constexpr (NTS == 2) {
#pragma unroll
            for (int v = 0; v < M; ++v) {
                const R other = __shfl_xor_sync(0xffffffffu, F[v], 1);
                if (isSub && t == 0) sF[v][f] = (F[v] + other) * R(0.5);
                else if (act && !isSub) sF[v][f] = F[v];
            }
        } else if constexpr (NTS == 4) {
#pragma unroll
            for (int v = 0; v < M; ++v) {
                const R pair = F[v] + __shfl_xor_sync(0xffffffffu, F[v], 1);
                const R quad = pair + __shfl_xor_sync(0xffffffffu, pair, 2);
                if (isSub && t == 0) sF[v][f] = quad * R(0.25);
                else if (act && !isSub) sF[v][f] = F[v];
            }
        } else if (act) {
#pragma unroll
            for (int v = 0; v < M; ++v) sF[v][f] = F[v];
        }
    }
    __syncthreads();

    // 4. compact RK update of the tile's leaves (thread tid < NC owns cell tid)
    if (tid < S::NC) {
        const int i = tid % TX, j = D > 1 ? (tid / TX) % TY : 0, kz = D > 2 ? tid / (TX * TY) : 0;
        const int bx = H + i, by = D > 1 ? H + j : 0, bz = D > 2 ? H + kz : 0;
        const int b = bz * SZ + by * SY + bx;
        if (tile_leaf(bx, by, bz)) {
        const long long id = cell_id(g, u, ox + i, oy + j, oz + kz);
        double self[M], f[M], q0p[M];
#pragma unroll
        for (int v = 0; v < M; ++v) self[v] = sW[v][b];
        if (s >= 2) { // q^n (the stage value itself is the staged exposure)
            const long long N = g.N[u];
            const double* q0 = fbase(g, F_Q0, u) + id;
#pragma unroll
            for (int v = 0; v < M; ++v) q0p[v] = q0[v * N];
        } else {
#pragma unroll
            for (int v = 0; v < M; ++v) q0p[v] = self[v];
        }
        source<EQ, M>(g, self, f);
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const int stride = k == 0 ? 1 : (k == 1 ? SY : SZ);
            const int bm = b - stride, bp = b + stride;
            int fm, fp;
            if (k == 0) {
                fm = i + (TX + 1) * (j + TY * kz);
                fp = fm + 1;
            } else if (k == 1) {
                fm = NFX + i + TX * (j + (TY + 1) * kz);
                fp = fm + TX;
            } else {
                fm = NFX + NFY + i + TX * (j + TY * kz);
                fp = fm + TX * TY;
            }
            const int sm = sSt[bm], sp = sSt[bp];
            const int km = (sm == 2 && finer) ? K_FINER : (sm == 1 ? K_LEAF : (sm == OUT ? K_WALL : K_COARSER));
            const int kp = (sp == 2 && finer) ? K_FINER : (sp == 1 ? K_LEAF : (sp == OUT ? K_WALL : K_COARSER));
            double Fm[M], Fp[M];
#pragma unroll
            for (int v = 0; v < M; ++v) {
                Fm[v] = double(sF[v][fm]);
                Fp[v] = double(sF[v][fp]);
            }
            const double idx = g.rdx[u][k];
#pragma unroll
            for (int v = 0; v < M; ++v) f[v] += (Fm[v] - Fp[v]) * idx;
            if (reg) {
                reg_add<M>(g, u, id, 2 * k, km, bw, Fm);
                reg_add<M>(g, u, id, 2 * k + 1, kp, bw, Fp);
            }
        }
        rk_update<M>(g, u, id, s, dtl, f, q0p, self);
        }
    }
    __syncthreads(); // shared arrays are reused by the next tile
    }
}

static inline int grid_for(const Grid& g, int l)
{
    long long b = (g.N[l] + NTHREADS - 1) / NTHREADS;
    return (int)(b < 1216 ? (b < 1 ? 1 : b) : 1216);
}

// One launch of the tiled stage kernel over the active tiles of levels lo..hi;
// the persistent grid is the device's resident capacity for this instantiation
// (occupancy API, once per device), capped by the tile count and by g.gcap
// when that is set.  CTAs stride over the tile slots and every cell's update
// and flux registers are written by one thread, so the result does not depend
// on the grid size.
template <int EQ, int D, class R>
static int stage_dispatch(const Grid& g, cudaStream_t st, int lo, int hi, int s, int lmin, double b, int reg)
{
    using S = TileShape<EQ, D, R>;
    constexpr int kMaxDev = 64;
    static int resident[kMaxDev] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return -1;
    if (!resident[dev]) {
        if (cudaFuncSetAttribute(k_stage_tile<EQ, D, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)S::SMEM) != cudaSuccess)
            return -1;
        int per_sm = 0, sms = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_stage_tile<EQ, D, R>, S::NT, S::SMEM) !=
                cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || per_sm < 1)
            return -1;
        resident[dev] = per_sm * sms;
    }
    if (lo > hi) return 0; // set-up only
    long long total = 0;
    for (int l = lo; l <= hi; ++l) total += (long long)g.ntx[l] * g.nty[l] * g.ntz[l];
    long long grid = total < resident[dev] ? total : resident[dev];
    if (g.gcap > 0 && grid > g.gcap) grid = g.gcap;
    if (grid < 1) grid = 1;
    // launched without a programmatic dependency: the persistent grid assigns
    // tiles statically, so it must find the SMs free to be resident at once
    k_stage_tile<EQ, D, R><<<(unsigned)grid, S::NT, S::SMEM, st>>>(g, lo, hi, s, lmin, b, reg);
    return 1;
}

// stage launcher of one equation (all dimensions, both precisions); each is
// defined in its own translation unit so that they compile in parallel
template <int EQ>
int launch_stage_eq(const Grid& g, cudaStream_t st, int lo, int hi, int s, int lmin, double b, int reg);
template <> int launch_stage_eq<0>(const Grid&, cudaStream_t, int, int, int, int, double, int);
template <> int launch_stage_eq<1>(const Grid&, cudaStream_t, int, int, int, int, double, int);
template <> int launch_stage_eq<2>(const Grid&, cudaStream_t, int, int, int, int, double, int);
template <> int launch_stage_eq<3>(const Grid&, cudaStream_t, int, int, int, int, double, int);

} // namespace mrlt

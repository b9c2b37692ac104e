// mrlt_stage.cuh -- the stage kernels of the MR/MRLT time evolution: face
// fluxes from the exposures of Secs. 4.1-4.3, the compact RK update of Sec. 3
// and the flux-register epilogue.
//  - k_stage_tile (d = 1, 2): one CTA per tile of one level; the halo is
//    staged in shared memory and every face flux is computed once.
//  - k_stage (d = 3): one thread per leaf.
// Both are instantiated for R = double and, for the mixed-precision mode, for
// R = float: reconstruction and numerical flux in R; the stored state, the
// right-hand side, the RK update and the flux registers stay in double.
#pragma once
#include "mrlt_impl.cuh"

namespace mrlt {

// Face flux of the leaf at c (level u) in direction k, side -1/+1, oriented
// along +x_k (Sec. 2 flux scenarios).  Returns the face kind.
template <int EQ, int D, int M, class R>
__device__ __forceinline__ int face_flux(const Grid& g, const Ctx& x, int u, const int c[3], int k,
                                         int side, double* F)
{
    int kind, q;
    bool sub = false;
    if (!in_box(g, u, k, c[k] + side, &q)) {
        kind = K_WALL;
    } else {
        int nb[3] = {c[0], c[1], c[2]};
        nb[k] = q;
        const int s = status(g, u, cell_id(g, u, nb[0], nb[1], nb[2]));
        if (s == 2 && u < g.L) {
            sub = true;
            kind = K_FINER;
        } else {
            kind = s == 1 ? K_LEAF : K_COARSER;
        }
    }
    double W[4][M];
    if (!sub) {
        int p[3] = {c[0], c[1], c[2]};
        const int first = side > 0 ? c[k] - 1 : c[k] - 2;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            p[k] = first + i;
            value_at<D, M>(g, x, u, p, W[i]);
        }
        R Fr[M];
        num_flux<EQ, D, M, R>(g, k, g.dx[u][k], W, Fr);
#pragma unroll
        for (int v = 0; v < M; ++v) F[v] = double(Fr[v]);
        return kind;
    }
    // internal neighbour: mean of the 2^{d-1} sub-face fluxes on level u+1
    constexpr int NT = 1 << (D - 1);
    double acc[M];
#pragma unroll
    for (int v = 0; v < M; ++v) acc[v] = 0.0;
#pragma unroll 1
    for (int t = 0; t < NT; ++t) {
        int p[3] = {0, 0, 0}, bit = 0;
#pragma unroll
        for (int j = 0; j < D; ++j) {
            if (j == k) continue;
            p[j] = 2 * c[j] + ((t >> bit) & 1);
            ++bit;
        }
        const int first = side > 0 ? 2 * c[k] : 2 * c[k] - 2;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            p[k] = first + i;
            value_at<D, M>(g, x, u + 1, p, W[i]);
        }
        R Fs[M];
        num_flux<EQ, D, M, R>(g, k, g.dx[u + 1][k], W, Fs);
#pragma unroll
        for (int v = 0; v < M; ++v) acc[v] += double(Fs[v]);
    }
#pragma unroll
    for (int v = 0; v < M; ++v) F[v] = acc[v] * (1.0 / NT);
    return kind;
}

// Compact RK update of one leaf from its right-hand side f (Sec. 3):
//   s = 1: q*  = q^n + dt_l f
//   s = 2: RK2 q^{n+1} = q^n/2 + q*/2 + dt_l f/2 ; RK3 q** = 3q^n/4 + q*/4 + dt_l f/4
//   s = 3: q^{n+1} = q^n/3 + 2q**/3 + 2 dt_l f/3
template <int M>
__device__ __forceinline__ void rk_update(const Grid& g, int u, long long id, int s, double dtl, const double* f)
{
    const long long N = g.N[u];
    double* q0 = fbase_w(g, F_Q0, u) + id;
    double* q1 = fbase_w(g, F_Q1, u) + id;
    double* q2 = fbase_w(g, F_Q2, u) + id;
    double* qe = fbase_w(g, F_QE, u) + id;
#pragma unroll
    for (int v = 0; v < M; ++v) {
        const double kk = dtl * f[v];
        if (s == 1) {
            q1[v * N] = q0[v * N] + kk;
        } else if (s == 2) {
            if (g.rk == 2) qe[v * N] = 0.5 * q0[v * N] + 0.5 * q1[v * N] + 0.5 * kk;
            else q2[v * N] = 0.75 * q0[v * N] + 0.25 * q1[v * N] + 0.25 * kk;
        } else {
            qe[v * N] = (1.0 / 3.0) * q0[v * N] + (2.0 / 3.0) * q2[v * N] + (2.0 / 3.0) * kk;
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

// One compact RK stage of every leaf of level u, one thread per leaf (d = 3).
template <int EQ, int D, class R>
__global__ void __launch_bounds__(NTHREADS) k_stage(Grid g, int u, int s, int lmin, double dtl,
                                                    double bw, int reg)
{
    constexpr int M = EQ == 2 ? D + 2 : 1;
    const int cnt = g.counts[u];
    const int* list = g.leaves + g.off[u];
    const long long N = g.N[u];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (s == 1) atomicAdd(g.updates, (unsigned long long)cnt);
        atomicAdd(&g.work[u * 4 + s], (unsigned long long)cnt);
    }
    const Ctx x{u, s, lmin};
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += gridDim.x * blockDim.x) {
        const long long id = list[t];
        if (id < 0 || id >= N) {
            atomicOr(g.err, ERR_INDEX);
            continue;
        }
        int c[3];
        cell_xyz(g, u, id, c);
        double self[M], f[M];
        expose<M>(g, x, u, id, 1, self);
        source<EQ, M>(g, self, f);
#pragma unroll 1
        for (int k = 0; k < D; ++k) {
            double Fm[M], Fp[M];
            const int km = face_flux<EQ, D, M, R>(g, x, u, c, k, -1, Fm);
            const int kp = face_flux<EQ, D, M, R>(g, x, u, c, k, +1, Fp);
            const double idx = g.rdx[u][k];
#pragma unroll
            for (int v = 0; v < M; ++v) f[v] += (Fm[v] - Fp[v]) * idx;
            if (reg) {
                reg_add<M>(g, u, id, 2 * k, km, bw, Fm);
                reg_add<M>(g, u, id, 2 * k + 1, kp, bw, Fp);
            }
        }
        rk_update<M>(g, u, id, s, dtl, f);
    }
}

// Tile shapes of the tiled stage kernel: a CTA owns TX x TY cells of one level
// (the same shapes index the per-level active-tile lists).
template <int D> struct Tile;
template <> struct Tile<1> { static constexpr int TX = kTile1X, TY = 1; };
template <> struct Tile<2> { static constexpr int TX = kTile2X, TY = kTile2Y; };
// resident CTAs of a persistent stage launch (152 SMs x 3)
constexpr long long kStageCtas = 456;

// Append, in thread order, the items for which `take` holds to a shared list
// (warp ballots and a block-wide prefix); every thread of the block calls it
// with the same `len` and gets the new length.
template <int NT>
__device__ __forceinline__ int block_append(bool take, int item, short* list, int len, int* sWarp)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned bal = __ballot_sync(0xffffffffu, take);
    if (lane == 0) sWarp[warp] = __popc(bal);
    __syncthreads();
    int before = 0, total = 0;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) {
        const int c = sWarp[w];
        before += w < warp ? c : 0;
        total += c;
    }
    if (take) list[len + before + __popc(bal & ((1u << lane) - 1u))] = (short)item;
    __syncthreads();
    return len + total;
}

// Tiled stage (d = 1, 2).  The CTA
//  1. reads the status of its tile and a 2-cell ring; tiles without leaves exit;
//  2. lists the cells some leaf of the tile reads -- its radius-2 cross stencil,
//     plus the 3^d block of a leaf facing an internal node -- and stages their
//     exposures (Secs. 4.1-4.3) and reconstruction variables in shared memory,
//     stored nodes first, then virtual cells and ghosts;
//  3. lists the faces touching a tile leaf and computes each once: plain faces
//     on level u from the shared cells; faces of a leaf against an internal node
//     as the mean of 2^{d-1} sub-face fluxes on level u+1 (Sec. 2), one thread
//     per sub-face, the leaf's virtual children predicted (Eq. 4) from its
//     shared 3^d block and the finer side read from level u+1;
//  4. applies the compact RK update and the register epilogue to its leaves.
// Work lists keep every warp on one kind of work.
template <int EQ, int D, class R>
__global__ void __launch_bounds__(Tile<D>::TX * Tile<D>::TY)
k_stage_tile(Grid g, int lo, int hi, int s, int lmin, double dt, double bstage, int reg)
{
    constexpr int M = EQ == 2 ? D + 2 : 1;
    constexpr int TX = Tile<D>::TX, TY = Tile<D>::TY, NT = TX * TY, H = 2;
    constexpr int BX = TX + 2 * H, BY = D > 1 ? TY + 2 * H : 1, NB = BX * BY;
    constexpr int NFX = (TX + 1) * TY, NFY = D > 1 ? TX * (TY + 1) : 0, NF = NFX + NFY;
    constexpr int NTS = 1 << (D - 1); // sub-faces per face
    constexpr int NL = NB > NF ? NB : NF;
    constexpr int OUT = 3;            // status code of a cell past a wall
    __shared__ double sW[M][NB];
    __shared__ R sP[M][NB];
    __shared__ R sF[M][NF];           // x faces [0, NFX), y faces [NFX, NF)
    __shared__ uint8_t sSt[NB];
    __shared__ short sList[NL];
    __shared__ int sWarp[NT / 32];

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
    const int ntx = (n + TX - 1) / TX;
    const int ox = (tile % ntx) * TX;
    const int oy = D > 1 ? (tile / ntx) * TY : 0;
    const int tid = threadIdx.x;
    const Ctx x{u, s, lmin};
    const bool finer = u < g.L; // internal nodes of level u have children

    // is block cell (bx, by) a leaf of this tile?
    auto tile_leaf = [&](int bx, int by) -> bool {
        if (bx < H || bx >= H + TX || ox + bx - H >= n) return false;
        if (D > 1 && (by < H || by >= H + TY || oy + by - H >= n)) return false;
        return sSt[by * BX + bx] == 1;
    };
    // a tile leaf with an internal node across one of its faces
    auto leaf_li = [&](int bx, int by) -> bool {
        if (!finer || !tile_leaf(bx, by)) return false;
        const int b = by * BX + bx;
        bool li = sSt[b - 1] == 2 || sSt[b + 1] == 2;
        if (D > 1) li = li || sSt[b - BX] == 2 || sSt[b + BX] == 2;
        return li;
    };
    auto needed = [&](int b) -> bool {
        const int bx = b % BX, by = b / BX;
        bool need = false;
#pragma unroll
        for (int d = -2; d <= 2; ++d) {
            need = need || tile_leaf(bx + d, by);
            if (D > 1) need = need || tile_leaf(bx, by + d);
        }
#pragma unroll
        for (int dy = (D > 1 ? -1 : 0); dy <= (D > 1 ? 1 : 0); ++dy)
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) need = need || leaf_li(bx + dx, by + dy);
        return need;
    };
    // geometry of face f: the cells on its two sides and the direction
    auto face = [&](int f, int& k, int& lo, int& hi, bool& leafLo, bool& leafHi) {
        if (f < NFX) {
            const int i = f % (TX + 1), j = f / (TX + 1);
            const int by = D > 1 ? H + j : 0;
            k = 0;
            lo = by * BX + H + i - 1;
            hi = lo + 1;
            leafLo = tile_leaf(H + i - 1, by);
            leafHi = tile_leaf(H + i, by);
        } else {
            const int ff = f - NFX, i = ff % TX, j = ff / TX;
            k = 1;
            lo = (H + j - 1) * BX + H + i;
            hi = lo + BX;
            leafLo = tile_leaf(H + i, H + j - 1);
            leafHi = tile_leaf(H + i, H + j);
        }
    };

    // 1. status of the tile and its ring
    for (int b = tid; b < NB; b += NT) {
        const int bx = b % BX, by = b / BX;
        int qx, qy = 0;
        const bool inb = in_box(g, u, 0, ox + bx - H, &qx) && (D < 2 || in_box(g, u, 1, oy + by - H, &qy));
        sSt[b] = inb ? status(g, u, cell_id(g, u, qx, qy, 0)) : OUT;
    }
    __syncthreads();
    const int nleaf = __syncthreads_count(tile_leaf(H + tid % TX, D > 1 ? H + tid / TX : 0));
    if (nleaf == 0) continue; // uniform across the CTA
    if (tid == 0) {
        if (s == 1) atomicAdd(g.updates, (unsigned long long)nleaf);
        atomicAdd(&g.work[u * 4 + s], (unsigned long long)nleaf);
    }

    // 2. exposures of the needed cells: stored nodes, then the others
    int nst = 0;
    for (int b0 = 0; b0 < NB; b0 += NT) {
        const int b = b0 + tid;
        nst = block_append<NT>(b < NB && (sSt[b] == 1 || sSt[b] == 2) && needed(b), b, sList, nst, sWarp);
    }
    int ncell = nst;
    for (int b0 = 0; b0 < NB; b0 += NT) {
        const int b = b0 + tid;
        ncell = block_append<NT>(b < NB && sSt[b] != 1 && sSt[b] != 2 && needed(b), b, sList, ncell, sWarp);
    }
    for (int t = tid; t < ncell; t += NT) {
        const int b = sList[t];
        const int bx = b % BX, by = b / BX;
        double W[M];
        R P[M];
        if (t < nst) {
            int qx, qy = 0;
            in_box(g, u, 0, ox + bx - H, &qx);
            if (D > 1) in_box(g, u, 1, oy + by - H, &qy);
            expose<M>(g, x, u, cell_id(g, u, qx, qy, 0), sSt[b], W);
        } else {
            const int p[3] = {ox + bx - H, D > 1 ? oy + by - H : 0, 0};
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

    // 3a. plain faces on level u
    int nfl = 0;
    for (int f0 = 0; f0 < NF; f0 += NT) {
        const int f = f0 + tid;
        bool take = false;
        if (f < NF) {
            int k, lo, hi;
            bool lL, lH;
            face(f, k, lo, hi, lL, lH);
            const bool sub = finer && ((lL && sSt[hi] == 2) || (lH && sSt[lo] == 2));
            take = (lL || lH) && !sub;
        }
        nfl = block_append<NT>(take, f, sList, nfl, sWarp);
    }
    for (int t = tid; t < nfl; t += NT) {
        const int f = sList[t];
        int k, lo, hi;
        bool lL, lH;
        face(f, k, lo, hi, lL, lH);
        const int stride = k == 0 ? 1 : BX;
        R F[M];
        flux_recon<EQ, D, M, R>(g, k, g.dx[u][k], [&](int c, int v) { return sP[v][lo + (c - 1) * stride]; }, F);
#pragma unroll
        for (int v = 0; v < M; ++v) sF[v][f] = F[v];
    }
    __syncthreads();

    // 3b. faces of a leaf against an internal node: one thread per sub-face
    int nsb = 0;
    if (finer) {
        for (int f0 = 0; f0 < NF; f0 += NT) {
            const int f = f0 + tid;
            bool take = false;
            if (f < NF) {
                int k, lo, hi;
                bool lL, lH;
                face(f, k, lo, hi, lL, lH);
                take = (lL && sSt[hi] == 2) || (lH && sSt[lo] == 2);
            }
            nsb = block_append<NT>(take, f, sList, nsb, sWarp);
        }
    }
    for (int base = 0; base < nsb * NTS; base += NT) {
        const int task = base + tid;
        const bool act = task < nsb * NTS;
        const int f = act ? sList[task / NTS] : 0, t = task % NTS;
        R F[M];
#pragma unroll
        for (int v = 0; v < M; ++v) F[v] = R(0);
        if (act) {
            int k, lo, hi;
            bool lL, lH;
            face(f, k, lo, hi, lL, lH);
            const bool leafIsLo = lL && sSt[hi] == 2;
            const int bl = leafIsLo ? lo : hi, side = leafIsLo ? 1 : -1;
            const int bx = bl % BX, by = bl / BX;
            const int c0 = ox + bx - H, c1 = D > 1 ? oy + by - H : 0;
            R P4[4][M];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                // stencil cell i on level u+1: fine coordinate along k and along
                // the face; the leaf's own children are virtual
                const int fk = (k == 0 ? 2 * c0 : 2 * c1) + (side > 0 ? i : i - 2);
                const int ft = (k == 0 ? 2 * c1 : 2 * c0) + t;
                const bool own = side > 0 ? i < 2 : i >= 2;
                double W[M];
                if (own) {
                    const int ax = k == 0 ? (fk & 1) : (ft & 1);
                    const int ay = k == 0 ? (ft & 1) : (fk & 1);
#pragma unroll
                    for (int v = 0; v < M; ++v) W[v] = 0.0;
#pragma unroll
                    for (int dy = (D > 1 ? -1 : 0); dy <= (D > 1 ? 1 : 0); ++dy)
#pragma unroll
                        for (int dx = -1; dx <= 1; ++dx) {
                            const double w = (D > 1 ? pw(ay, dy) : 1.0) * pw(ax, dx);
                            const int bs = (by + dy) * BX + bx + dx;
#pragma unroll
                            for (int v = 0; v < M; ++v) W[v] += w * sW[v][bs];
                        }
                } else {
                    int p[3] = {0, 0, 0};
                    p[k] = fk;
                    if (D > 1) p[1 - k] = ft;
                    value_at<D, M>(g, x, u + 1, p, W);
                }
                recon_vars<EQ, D, M, R>(g, W, P4[i]);
            }
            flux_recon<EQ, D, M, R>(g, k, g.dx[u + 1][k], [&](int c, int v) { return P4[c][v]; }, F);
        }
        if constexpr (NTS == 2) { // the two sub-faces of a face sit in lanes 2i, 2i+1
#pragma unroll
            for (int v = 0; v < M; ++v) {
                const R other = __shfl_xor_sync(0xffffffffu, F[v], 1);
                if (act && t == 0) sF[v][f] = (F[v] + other) * R(0.5);
            }
        } else if (act) {
#pragma unroll
            for (int v = 0; v < M; ++v) sF[v][f] = F[v];
        }
    }
    __syncthreads();

    // 4. compact RK update of the tile's leaves
    {
        const int i = tid % TX, j = D > 1 ? tid / TX : 0;
        const int bx = H + i, by = D > 1 ? H + j : 0, b = by * BX + bx;
        if (tile_leaf(bx, by)) {
        const long long id = cell_id(g, u, ox + i, oy + j, 0);
        double self[M], f[M];
#pragma unroll
        for (int v = 0; v < M; ++v) self[v] = sW[v][b];
        source<EQ, M>(g, self, f);
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const int bm = k == 0 ? b - 1 : b - BX, bp = k == 0 ? b + 1 : b + BX;
            const int fm = k == 0 ? j * (TX + 1) + i : NFX + j * TX + i;
            const int fp = k == 0 ? fm + 1 : fm + TX;
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
        rk_update<M>(g, u, id, s, dtl, f);
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

template <int EQ, int D, class R>
static int stage_dispatch(const Grid& g, cudaStream_t st, int lo, int hi, int s, int lmin, double dt,
                          double b, int reg)
{
    if constexpr (D <= 2) {
        long long total = 0;
        for (int l = lo; l <= hi; ++l) total += (long long)g.ntx[l] * g.nty[l];
        const long long grid = total < kStageCtas ? total : kStageCtas;
        k_stage_tile<EQ, D, R><<<(unsigned)grid, Tile<D>::TX * Tile<D>::TY, 0, st>>>(g, lo, hi, s, lmin, dt, b, reg);
        return 1;
    } else {
        for (int u = lo; u <= hi; ++u) {
            const double dtl = g.gts ? dt : ldexp(dt, g.L - u);
            k_stage<EQ, D, R><<<grid_for(g, u), NTHREADS, 0, st>>>(g, u, s, lmin, dtl, dtl * b, reg);
        }
        return hi - lo + 1;
    }
}

// stage launcher of one equation (all dimensions, both precisions); each is
// defined in its own translation unit so that they compile in parallel
template <int EQ>
int launch_stage_eq(const Grid& g, cudaStream_t st, int lo, int hi, int s, int lmin, double dt, double b,
                    int reg);
template <> int launch_stage_eq<0>(const Grid&, cudaStream_t, int, int, int, int, double, double, int);
template <> int launch_stage_eq<1>(const Grid&, cudaStream_t, int, int, int, int, double, double, int);
template <> int launch_stage_eq<2>(const Grid&, cudaStream_t, int, int, int, int, double, double, int);
template <> int launch_stage_eq<3>(const Grid&, cudaStream_t, int, int, int, int, double, double, int);

} // namespace mrlt

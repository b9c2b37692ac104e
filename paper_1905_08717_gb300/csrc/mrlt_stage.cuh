// mrlt_stage.cuh -- the stage kernels of the MR/MRLT time evolution: face
// fluxes from the exposures of Secs. 4.1-4.3, the compact RK update of Sec. 3
// and the flux-register epilogue.
// k_stage_tile (d = 1, 2, 3) works on one tile of one level per CTA: the
// halo is staged in shared memory and every face flux is computed once.  It is
// instantiated for R = double and, for the mixed-precision mode, R = float:
// the stored state, the exposures, the reconstruction, the numerical fluxes,
// the right-hand side and the RK update are all in R; the flux registers
// accumulate in double.
#pragma once
#include "mrlt_impl.cuh"

namespace mrlt {

// Compact RK update of one leaf from its right-hand side f (Sec. 3):
//   s = 1: q*  = q^n + dt_l f
//   s = 2: RK2 q^{n+1} = q^n/2 + q*/2 + dt_l f/2 ; RK3 q** = 3q^n/4 + q*/4 + dt_l f/4
//   s = 3: q^{n+1} = q^n/3 + 2q**/3 + 2 dt_l f/3
// qs is the leaf's own value at stage s (q^n, q*, q** for s = 1, 2, 3: its
// exposure, already staged in shared memory) and q0 its q^n (s >= 2).
template <int M, class R>
__device__ __forceinline__ void rk_update(const Grid& g, int sl, int s, R dtl, const R* f, const R* q0, const R* qs)
{
    R* q1 = nd<R>(g, F_Q1, sl);
    R* q2 = nd<R>(g, F_Q2, sl);
    R* qe = nd<R>(g, F_QE, sl);
#pragma unroll
    for (int v = 0; v < M; ++v) {
        const R kk = dtl * f[v];
        if (s == 1) {
            q1[v] = qs[v] + kk;
        } else if (s == 2) {
            if (g.rk == 2) qe[v] = R(0.5) * q0[v] + R(0.5) * qs[v] + R(0.5) * kk;
            else q2[v] = R(0.75) * q0[v] + R(0.25) * qs[v] + R(0.25) * kk;
        } else {
            qe[v] = R(1.0 / 3.0) * q0[v] + R(2.0 / 3.0) * qs[v] + R(2.0 / 3.0) * kk;
        }
    }
}

// flux registers (conservation across levels): dt_l b_s F at coarse-fine faces
template <int M>
__device__ __forceinline__ void reg_add(const Grid& g, int sl, int fi, int kind, double bw, const double* F)
{
    if (kind != K_FINER && kind != K_COARSER) return;
    double* R = regs(g.rg, g, sl); // coarse side (K_FINER) or fine side (K_COARSER) of the face
#pragma unroll
    for (int v = 0; v < M; ++v) R[fi * M + v] += bw * F[v];
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
    // parent-level block: the cells of level u-1 whose exposures predict the
    // virtual cells of the block (Eq. 4 reads a 3^d neighbourhood of the parent)
    static constexpr int PBX = TX / 2 + 4, PBY = D > 1 ? TY / 2 + 4 : 1, PBZ = D > 2 ? TZ / 2 + 4 : 1;
    static constexpr int PB = PBX * PBY * PBZ;
    // sub-face tasks whose two finer-side cells are fetched with the exposures
    static constexpr int NPF = D > 2 ? 64 : NT;
    // dynamic shared memory (all R): conservative values of the block, of the
    // parent block and q^n of the tile, reconstruction variables, face fluxes
    // and the prefetched finer-side variables
    static constexpr size_t SMEM = sizeof(R) * M * (2 * NB + PB + NC + NF + 2 * NPF);
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

// Value of the stored finer-level node at in-box coordinates q of level l =
// u + 1 as the level-u stencil sees it at stage x.s (the rel = +1 rows of
// expose()): its status and slot, then every field the choice may need,
// loaded at once.  Returns false (out untouched) when the cell is absent.
template <int M, class T>
__device__ __forceinline__ bool finer_exposure(const Grid& g, const Ctx& x, int l, const int q[3], T* out)
{
    const long long id = cell_id(g, l, q[0], q[1], q[2]);
    const int st = status(g, l, id);
    const int sl = slot_of(g, l, id);
    const T* q0 = nd<T>(g, F_Q0, sl);
    if (x.s <= 1) {
        T a[M];
#pragma unroll
        for (int v = 0; v < M; ++v) a[v] = q0[v];
        if (st == 0) return false;
#pragma unroll
        for (int v = 0; v < M; ++v) out[v] = a[v];
        return true;
    }
    if (g.gts || x.s == 3) { // global step: q* / q**; LT stage 3: q^{n+1} of the first sub-step
        const T* a = nd<T>(g, g.gts ? (x.s == 2 ? F_Q1 : F_Q2) : F_QE, sl);
        T b[M];
#pragma unroll
        for (int v = 0; v < M; ++v) b[v] = a[v];
        if (st == 0) return false;
#pragma unroll
        for (int v = 0; v < M; ++v) out[v] = b[v];
        return true;
    }
    // LT stage 2: leaf Eq. 14 (q* + k2), internal node Eq. 15 (2 q* - q^n)
    const T* q1 = nd<T>(g, F_Q1, sl);
    const T* qx = nd<T>(g, g.rk == 2 ? F_QE : F_Q2, sl);
    T a0[M], a1[M], ax[M];
#pragma unroll
    for (int v = 0; v < M; ++v) {
        a0[v] = q0[v];
        a1[v] = q1[v];
        ax[v] = qx[v];
    }
    if (st == 0) return false;
    if (st == 1) {
        if (g.rk == 2) {
#pragma unroll
            for (int v = 0; v < M; ++v) out[v] = T(2) * ax[v] - a0[v];
        } else {
#pragma unroll
            for (int v = 0; v < M; ++v) out[v] = T(4) * ax[v] - T(3) * a0[v];
        }
    } else {
#pragma unroll
        for (int v = 0; v < M; ++v) out[v] = T(2) * a1[v] - a0[v];
    }
    return true;
}

// Tiled stage (d = 1, 2, 3).  The CTA works on one tile of one level at a
// time, in phases separated by CTA barriers, with as few dependent trips to
// memory as the data allow:
//  1. status of the tile, its 2-cell ring and the parent-level block (one
//     trip); tiles without leaves are skipped;
//  2. lists, from the statuses alone: the cells some tile leaf reads -- its
//     radius-2 cross stencil and the 3^d block of a leaf facing an internal
//     node -- split into stored nodes and virtual cells (absent nodes and
//     ghosts past a wall); the parent-block cells the virtual cells'
//     predictions (Eq. 4) read; the faces touching a tile leaf, split into
//     faces against an internal node (2^{d-1} sub-faces on level u+1, Sec. 2)
//     and plain faces;
//  3. one trip for everything the stage reads from memory: exposures
//     (Secs. 4.1-4.3) of the stored cells and of the parent-block cells, the
//     finer-side cells of the sub-faces, and q^n of the tile's leaves;
//  4. virtual cells predicted in shared memory from the parent block (a ghost
//     whose mirror image is stored takes that image's value);
//  5. every face touching a tile leaf computed once, one thread per face or
//     sub-face (the 2^{d-1} threads of a face are adjacent lanes, combined by
//     shuffles), the leaf's own virtual children predicted from its shared
//     3^d block;
//  6. the compact RK update and the flux-register epilogue of the tile's leaves.
// Work lists keep every warp on one kind of work.  Each value is computed by
// the same operations in the same order as the direct definitions (expose,
// predict, value_at); only the place its inputs come from changes.
// The tiles of levels lo..hi are distributed over the CTAs of the launch
// (blockIdx / gridDim); smem is the dynamic shared memory of TileShape::SMEM
// bytes.  Called by k_stage_tile and by the persistent macro-step kernel.
template <int EQ, int D, class R>
__device__ __forceinline__ void stage_tiles(const Grid& g, int lo, int hi, int s, int lmin, double bstage, int reg,
                                            unsigned char* smem)
{
    const double dt = *g.dtp; // fine step of the macro step
    using S = TileShape<EQ, D, R>;
    constexpr int M = S::M, TX = S::TX, TY = S::TY, TZ = S::TZ, NT = S::NT, H = S::H, NC = S::NC;
    constexpr int BX = S::BX, BY = S::BY, BZ = S::BZ, NB = S::NB;
    constexpr int NFX = S::NFX, NFY = S::NFY, NF = S::NF;
    constexpr int PBX = S::PBX, PBY = S::PBY, PBZ = S::PBZ, PB = S::PB, NPF = S::NPF;
    constexpr int NTS = 1 << (D - 1); // sub-faces per face
    constexpr int OUT = 3;            // status code of a cell past a wall
    constexpr int SY = BX, SZ = BX * BY;     // block strides in y and z
    constexpr int PSY = PBX, PSZ = PBX * PBY; // parent-block strides
    R (*sW)[NB] = reinterpret_cast<R (*)[NB]>(smem);
    R (*sPW)[PB] = reinterpret_cast<R (*)[PB]>(smem + sizeof(R) * M * NB);
    R (*sQ0)[NC] = reinterpret_cast<R (*)[NC]>(smem + sizeof(R) * M * (NB + PB));
    unsigned char* rbase = smem + sizeof(R) * M * (NB + PB + NC);
    R (*sP)[NB] = reinterpret_cast<R (*)[NB]>(rbase);
    // x faces [0, NFX), y faces [NFX, NFX + NFY), z faces [NFX + NFY, NF)
    R (*sF)[NF] = reinterpret_cast<R (*)[NF]>(rbase + sizeof(R) * M * NB);
    R (*sFine)[M][NPF] = reinterpret_cast<R (*)[M][NPF]>(rbase + sizeof(R) * M * (NB + NF));
    __shared__ uint8_t sSt[NB], sNeed[NB];  // status; needed | stored << 1
    __shared__ int sSlot[NB];               // node slots of the block cells
    __shared__ uint8_t sPSt[PB], sPNeg[PB], sPNeed[PB];
    __shared__ int sPSlot[PB];
    __shared__ short sList[NB], sList2[NB]; // stored, virtual cells
    __shared__ short sFace1[NF], sFace2[NF]; // faces against an internal node, plain faces
    __shared__ short sPList[PB];
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
    const bool finer = u < g.L;   // internal nodes of level u have children
    const bool pstage = u > g.lb; // a parent level exists
    // parent-block origin (level u-1 coordinates, before wrapping)
    const int pox = (ox >> 1) - 2, poy = D > 1 ? (oy >> 1) - 2 : 0, poz = D > 2 ? (oz >> 1) - 2 : 0;

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
    // A virtual cell b: coordinates p (possibly past a wall); the in-box cell
    // q that value_at() reads instead (wrapped or mirrored, neg = its value
    // enters negated); the block cell bq holding q's status (-1: outside the
    // block); the parent-block index pb0 of the corner of the 3^d
    // neighbourhood whose exposures predict q (-1: outside the parent block).
    // In a periodic direction the block cell itself holds the wrapped status,
    // and the parent neighbourhood of p >> 1 wraps onto that of q >> 1.
    auto resolve = [&](int b, int p[3], int q[3], int& neg, int& bq, int& pb0) {
        const int bc3[3] = {b % BX, (b / BX) % BY, b / SZ};
        const int o3[3] = {ox, oy, oz}, B3[3] = {BX, BY, BZ}, bs3[3] = {1, SY, SZ};
        const int po3[3] = {pox, poy, poz}, P3[3] = {PBX, PBY, PBZ}, ps3[3] = {1, PSY, PSZ};
        neg = 0;
        bq = 0;
        pb0 = 0;
        bool inb = true, inp = true;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            if (k >= D) {
                p[k] = q[k] = 0;
                continue;
            }
            p[k] = o3[k] + bc3[k] - H;
            q[k] = wrap_or_mirror(g, u, k, p[k], neg);
            const int bk = g.bc[k] == 0 ? bc3[k] : q[k] - o3[k] + H;
            inb = inb && bk >= 0 && bk < B3[k];
            bq += bk * bs3[k];
            const int pk = ((g.bc[k] == 0 ? p[k] : q[k]) >> 1) - 1 - po3[k];
            inp = inp && pk >= 0 && pk + 2 < P3[k];
            pb0 += pk * ps3[k];
        }
        if (!inb) bq = -1;
        if (!inp || !pstage) pb0 = -1;
    };

    // 1. status of the tile, its ring and the parent-level block
    for (int b = tid; b < NB; b += NT) {
        const int bx = b % BX, by = (b / BX) % BY, bz = b / SZ;
        int qx, qy = 0, qz = 0;
        const bool inb = in_box(g, u, 0, ox + bx - H, &qx) && (D < 2 || in_box(g, u, 1, oy + by - H, &qy)) &&
                         (D < 3 || in_box(g, u, 2, oz + bz - H, &qz));
        const long long id = cell_id(g, u, qx, qy, qz);
        sSt[b] = inb ? status(g, u, id) : OUT;
        sSlot[b] = inb ? slot_of(g, u, id) : -1;
    }
    if (pstage)
        for (int pb = tid; pb < PB; pb += NT) {
            const int i = pb % PBX, j = (pb / PBX) % PBY, kk = pb / PSZ;
            int neg = 0;
            const int px = wrap_or_mirror(g, u - 1, 0, pox + i, neg);
            const int py = D > 1 ? wrap_or_mirror(g, u - 1, 1, poy + j, neg) : 0;
            const int pz = D > 2 ? wrap_or_mirror(g, u - 1, 2, poz + kk, neg) : 0;
            const long long pid = cell_id(g, u - 1, px, py, pz);
            sPSt[pb] = status(g, u - 1, pid);
            sPSlot[pb] = slot_of(g, u - 1, pid);
            sPNeg[pb] = (uint8_t)neg;
            sPNeed[pb] = 0;
        }
    __syncthreads();
    const int nleaf = __syncthreads_count(
        tid < NC && tile_leaf(H + tid % TX, D > 1 ? H + (tid / TX) % TY : 0, D > 2 ? H + tid / (TX * TY) : 0));
    if (nleaf == 0) continue; // uniform across the CTA
    if (tid == 0) {
        if (s == 1) atomicAdd(g.updates, (unsigned long long)nleaf);
        atomicAdd(&g.work[u * 4 + s], (unsigned long long)nleaf);
    }

    // 2. lists: stored and virtual needed cells, parent cells, faces
    int nst = 0, nvc = 0, par = 0;
    for (int b0 = 0; b0 < NB; b0 += NT) {
        const int b = b0 + tid;
        const bool nd = b < NB && needed(b);
        const bool stored = nd && (sSt[b] == 1 || sSt[b] == 2);
        if (b < NB) sNeed[b] = (uint8_t)(nd | (stored << 1));
        block_append2<NT>(stored, nd && !stored, b, sList, sList2, nst, nvc, sWarp, par);
    }
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
        block_append2<NT>(sub, plain, f, sFace1, sFace2, nsb, nfl, sWarp, par);
    }
    __syncthreads(); // virtual list complete: mark the parent cells it reads
    for (int t = tid; t < nvc; t += NT) {
        int p[3], q[3], neg, bq, pb0;
        resolve(sList2[t], p, q, neg, bq, pb0);
        if (bq >= 0 && sSt[bq] == 0 && pb0 >= 0)
#pragma unroll
            for (int dz = 0; dz < (D > 2 ? 3 : 1); ++dz)
#pragma unroll
                for (int dy = 0; dy < (D > 1 ? 3 : 1); ++dy)
#pragma unroll
                    for (int dx = 0; dx < 3; ++dx) sPNeed[pb0 + dz * PSZ + dy * PSY + dx] = 1;
    }
    __syncthreads();
    int npl = 0, nnone = 0;
    if (pstage) {
        for (int p0 = 0; p0 < PB; p0 += NT) {
            const int pb = p0 + tid;
            block_append2<NT>(pb < PB && sPNeed[pb], false, pb, sPList, sPList, npl, nnone, sWarp, par);
        }
    }
    __syncthreads();
    const int nsub = nsb * NTS; // sub-face tasks come first; NTS divides 32

    // 3. one trip: exposures of stored and parent cells, finer-side cells of
    //    the first sub-face tasks, q^n of the tile's leaves
    R q0r[M];
    const bool own_leaf = s >= 2 && tid < NC &&
                          tile_leaf(H + tid % TX, D > 1 ? H + (tid / TX) % TY : 0, D > 2 ? H + tid / (TX * TY) : 0);
    if (own_leaf) {
        const int b = (D > 2 ? H + tid / (TX * TY) : 0) * SZ + (D > 1 ? H + (tid / TX) % TY : 0) * SY + H + tid % TX;
        const R* q0 = nd<R>(g, F_Q0, sSlot[b]);
#pragma unroll
        for (int v = 0; v < M; ++v) q0r[v] = q0[v];
    }
    for (int t = tid; t < nst + npl; t += NT) {
        R W[M];
        if (t < nst) {
            const int b = sList[t];
            expose<M, R, R>(g, x, u, sSlot[b], sSt[b], W);
            R P[M];
            recon_vars<EQ, D, M, R>(g, W, P);
#pragma unroll
            for (int v = 0; v < M; ++v) {
                sW[v][b] = W[v];
                sP[v][b] = P[v];
            }
        } else {
            const int pb = sPList[t - nst];
            const int st = sPSt[pb];
            if (st == 0) continue; // predict() flags the absent source when it reads it
            expose<M, R, R>(g, x, u - 1, sPSlot[pb], st, W);
            // an odd-mirror ghost enters negated: (-w) v = w (-v) exactly
            const bool neg = sPNeg[pb] != 0;
#pragma unroll
            for (int v = 0; v < M; ++v) sPW[v][pb] = neg ? -W[v] : W[v];
        }
    }
    if (tid < nsub && tid < NPF) { // sub-face task tid: its two finer-side cells
        const int f = sFace1[tid / NTS], t = tid % NTS;
        int k, lo, hi;
        bool lL, lH;
        face(f, k, lo, hi, lL, lH);
        const bool leafIsLo = lL && sSt[hi] == 2;
        const int bl = leafIsLo ? lo : hi, side = leafIsLo ? 1 : -1;
        const int bx = bl % BX, by = (bl / BX) % BY, bz = bl / SZ;
        const int c[3] = {ox + bx - H, D > 1 ? oy + by - H : 0, D > 2 ? oz + bz - H : 0};
        const int j1 = k == 0 ? 1 : 0, j2 = k == 2 ? 1 : 2;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int i = side > 0 ? 2 + r : r; // the cells on the internal node's side
            int p[3] = {0, 0, 0};
            p[k] = 2 * c[k] + (side > 0 ? i : i - 2);
            if (D > 1) p[j1] = 2 * c[j1] + (t & 1);
            if (D > 2) p[j2] = 2 * c[j2] + (t >> 1);
            int q[3] = {0, 0, 0}, neg = 0;
#pragma unroll
            for (int kk = 0; kk < D; ++kk) q[kk] = wrap_or_mirror(g, u + 1, kk, p[kk], neg);
            R W[M];
            if (!finer_exposure<M, R>(g, x, u + 1, q, W)) {
                value_at<D, M, R, R>(g, x, u + 1, p, W); // absent: predicted (flags the missing source)
            } else if (neg) {
#pragma unroll
                for (int v = 0; v < M; ++v) W[v] = -W[v];
            }
            R P[M];
            recon_vars<EQ, D, M, R>(g, W, P);
#pragma unroll
            for (int v = 0; v < M; ++v) sFine[r][v][tid] = P[v];
        }
    }
    if (own_leaf)
#pragma unroll
        for (int v = 0; v < M; ++v) sQ0[v][tid] = q0r[v];
    __syncthreads();

    // 4. virtual cells: predicted from the parent block (the terms of
    //    predict() in its order), or a stored mirror image, else value_at()
    for (int t = tid; t < nvc; t += NT) {
        const int b = sList2[t];
        int p[3], q[3], neg, bq, pb0;
        resolve(b, p, q, neg, bq, pb0);
        R W[M];
        if (bq >= 0 && sSt[bq] == 0 && pb0 >= 0) {
#pragma unroll
            for (int v = 0; v < M; ++v) W[v] = R(0);
            const int a0 = q[0] & 1, a1 = q[1] & 1, a2 = q[2] & 1;
#pragma unroll(D > 2 ? 1 : 3)
            for (int dz = (D > 2 ? -1 : 0); dz <= (D > 2 ? 1 : 0); ++dz) {
                const R wz = D > 2 ? R(pw(a2, dz)) : R(1);
#pragma unroll(D > 2 ? 1 : 3)
                for (int dy = (D > 1 ? -1 : 0); dy <= (D > 1 ? 1 : 0); ++dy) {
                    const R wyz = wz * (D > 1 ? R(pw(a1, dy)) : R(1));
#pragma unroll
                    for (int dxx = -1; dxx <= 1; ++dxx) {
                        const int pb = pb0 + (D > 2 ? (dz + 1) * PSZ : 0) + (D > 1 ? (dy + 1) * PSY : 0) + dxx + 1;
                        if (sPSt[pb] == 0) {
                            atomicOr(g.err, ERR_SOURCE);
                            continue;
                        }
                        const R w0 = wyz * R(pw(a0, dxx));
#pragma unroll
                        for (int v = 0; v < M; ++v) W[v] += w0 * sPW[v][pb];
                    }
                }
            }
            if (neg) {
#pragma unroll
                for (int v = 0; v < M; ++v) W[v] = -W[v];
            }
        } else if (bq >= 0 && (sNeed[bq] & 2)) { // a ghost whose mirror image is a staged stored cell
#pragma unroll
            for (int v = 0; v < M; ++v) W[v] = neg ? -sW[v][bq] : sW[v][bq];
        } else {
            value_at<D, M, R, R>(g, x, u, p, W);
        }
        R P[M];
        recon_vars<EQ, D, M, R>(g, W, P);
#pragma unroll
        for (int v = 0; v < M; ++v) {
            sW[v][b] = W[v];
            sP[v][b] = P[v];
        }
    }
    __syncthreads();

    // 5. the faces touching a tile leaf, one pass: faces of a leaf against an
    //    internal node (2^{d-1} sub-face tasks each, in adjacent lanes), then
    //    plain faces on level u, one thread per face
    for (int base = 0; base < nsub + nfl; base += NT) {
        const int task = base + tid;
        const bool isSub = task < nsub, act = task < nsub + nfl;
        const int f = isSub ? sFace1[task / NTS] : (act ? sFace2[task - nsub] : 0);
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
                const bool pre = task < NPF; // finer side fetched in phase 3
                R P4[4][M];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    // stencil cell i on level u+1; the leaf's own children are virtual
                    int p[3] = {0, 0, 0};
                    p[k] = 2 * c[k] + (side > 0 ? i : i - 2);
                    if (D > 1) p[j1] = 2 * c[j1] + (t & 1);
                    if (D > 2) p[j2] = 2 * c[j2] + (t >> 1);
                    const bool own = side > 0 ? i < 2 : i >= 2;
                    if (own) {
                        R W[M];
                        const int ax = p[0] & 1, ay = p[1] & 1, az = p[2] & 1;
#pragma unroll
                        for (int v = 0; v < M; ++v) W[v] = R(0);
#pragma unroll
                        for (int dz = (D > 2 ? -1 : 0); dz <= (D > 2 ? 1 : 0); ++dz)
#pragma unroll
                            for (int dy = (D > 1 ? -1 : 0); dy <= (D > 1 ? 1 : 0); ++dy)
#pragma unroll
                                for (int dx = -1; dx <= 1; ++dx) {
                                    const R w = R((D > 2 ? pw(az, dz) : 1.0) * (D > 1 ? pw(ay, dy) : 1.0)) *
                                                R(pw(ax, dx));
                                    const int bs = bl + dz * SZ + dy * SY + dx;
#pragma unroll
                                    for (int v = 0; v < M; ++v) W[v] += w * sW[v][bs];
                                }
                        recon_vars<EQ, D, M, R>(g, W, P4[i]);
                    } else if (pre) {
                        const int r = side > 0 ? i - 2 : i;
#pragma unroll
                        for (int v = 0; v < M; ++v) P4[i][v] = sFine[r][v][task];
                    } else {
                        R W[M];
                        value_at<D, M, R, R>(g, x, u + 1, p, W);
                        recon_vars<EQ, D, M, R>(g, W, P4[i]);
                    }
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

    // 6. compact RK update of the tile's leaves (thread tid < NC owns cell tid)
    if (tid < NC) {
        const int i = tid % TX, j = D > 1 ? (tid / TX) % TY : 0, kz = D > 2 ? tid / (TX * TY) : 0;
        const int bx = H + i, by = D > 1 ? H + j : 0, bz = D > 2 ? H + kz : 0;
        const int b = bz * SZ + by * SY + bx;
        if (tile_leaf(bx, by, bz)) {
        const int sl = sSlot[b];
        R self[M], f[M], q0p[M];
#pragma unroll
        for (int v = 0; v < M; ++v) self[v] = sW[v][b];
#pragma unroll
        for (int v = 0; v < M; ++v) q0p[v] = s >= 2 ? sQ0[v][tid] : self[v]; // the stage value is the staged exposure
        source<EQ, M, R>(g, self, f);
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
            const R idx = R(g.rdx[u][k]);
#pragma unroll
            for (int v = 0; v < M; ++v) f[v] += (R(Fm[v]) - R(Fp[v])) * idx;
            if (reg) {
                reg_add<M>(g, sl, 2 * k, km, bw, Fm);
                reg_add<M>(g, sl, 2 * k + 1, kp, bw, Fp);
            }
        }
        rk_update<M, R>(g, sl, s, R(dtl), f, q0p, self);
        }
    }
    __syncthreads(); // shared arrays are reused by the next tile
    }
}

template <int EQ, int D, class R>
__global__ void __launch_bounds__(Tile<D>::THREADS)
k_stage_tile(const __grid_constant__ Grid g, int lo, int hi, int s, int lmin, double bstage, int reg)
{
    MRLT_ENTER(g);
    extern __shared__ __align__(16) unsigned char smem[];
    stage_tiles<EQ, D, R>(g, lo, hi, s, lmin, bstage, reg, smem);
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

// mrlt_tree_dev.cuh -- device bodies of the tree work of the MRLT library:
// projections and tree refreshing (Eqs. 3, 14-22; Algs. 3, 4, 6, 8, 9), the
// multiresolution adaptation (details Eq. 5, thresholding Alg. 2, graded
// closure Alg. 1), list compaction, conservative flux registers and the
// per-macro-step reductions.  Each body distributes its work over the
// launch's grid (grid-stride loops over blockIdx / gridDim), so the same body
// serves a kernel of its own (mrlt_tree.cu) and a phase of the persistent
// macro-step kernel (mrlt_macro.cuh).
#pragma once
#include "mrlt_impl.cuh"

namespace mrlt {

enum ProjMode { PM_Q0 = 0, PM_Q1, PM_Q2, PM_REF2, PM_PRJ2, PM_REF3, PM_PRJ3, PM_MID };

#define MRLT_GRID_STRIDE(i, n) \
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (long long)gridDim.x * blockDim.x)

// ------------------------------------------------------------ simple leaf copies
// T: storage type of the fields (double, or float in the mixed mode); the
// arithmetic of a body is in T except where it says otherwise
template <class T>
__device__ __forceinline__ void dev_leaf_copy(const Grid& g, int lo, int hi, int from, int to)
{
    for (int l = lo; l <= hi; ++l) {
        const int cnt = g.counts[l];
        const int* list = g.leaves + g.off[l];
        const long long N = g.N[l];
        MRLT_GRID_STRIDE(t, cnt)
        {
            const long long id = list[t];
            if (id < 0 || id >= N) {
                atomicOr(g.err, ERR_INDEX);
                continue;
            }
            const int sl = slot_of(g, l, id);
            const T* a = nd<T>(g, from, sl);
            T* b = nd<T>(g, to, sl);
            for (int v = 0; v < g.m; ++v) b[v] = a[v];
        }
    }
}

// ------------------------------------------------------------ projections
// Every internal node of level l combines its 2^d children (Eq. 3 mean):
//  PM_Q0 / PM_Q1 / PM_Q2: plain projection of that field (Alg. 3; GTS stages)
//  PM_REF2: Alg. 8 -- XH = mean q* (Eq. 17), q* = 2 XH - q^n (Eq. 18)
//  PM_PRJ2: Alg. 4 -- q* = mean(leaf: Eq. 14 value, internal: Eq. 15 value)
//  PM_REF3: Alg. 9 -- N1 = mean q**, N3 by Eq. 20, q** by Eq. 21
//  PM_PRJ3: Alg. 6 -- q** = mean(children at t^n + dt_{l+1}), end value
//           2 q** - q^n (Eq. 16 with the theta values implied by q**)
//  PM_MID:  Alg. 3 / Sec. 4.3 refresh of the mid-step level lmin-1
// one internal node (l, id): the projection of the given mode
template <int D, class T>
__device__ __forceinline__ void project_node(const Grid& g, int l, long long id, int mode)
{
    constexpr int NCH = 1 << D;
    int c[3];
    cell_xyz(g, l, id, c);
    int csl[NCH];
    uint8_t cst[NCH];
#pragma unroll
    for (int k = 0; k < NCH; ++k) {
        const long long ch = cell_id(g, l + 1, 2 * c[0] + (k & 1), D > 1 ? 2 * c[1] + ((k >> 1) & 1) : 0,
                                     D > 2 ? 2 * c[2] + ((k >> 2) & 1) : 0);
        cst[k] = status(g, l + 1, ch);
        csl[k] = slot_of(g, l + 1, ch);
    }
    const int sl = slot_of(g, l, id);
    T* q0 = nd<T>(g, F_Q0, sl);
    T* q1 = nd<T>(g, F_Q1, sl);
    T* q2 = nd<T>(g, F_Q2, sl);
    T* qe = nd<T>(g, F_QE, sl);
    for (int v = 0; v < g.m; ++v) {
        const int o = v;
        T acc = T(0);
#pragma unroll
        for (int k = 0; k < NCH; ++k) {
            const T* c0 = nd<T>(g, F_Q0, csl[k]);
            const T* c1 = nd<T>(g, F_Q1, csl[k]);
            const T* c2 = nd<T>(g, F_Q2, csl[k]);
            const T* ce = nd<T>(g, F_QE, csl[k]);
            const int oc = v;
            T w;
            switch (mode) {
            case PM_Q0: w = c0[oc]; break;
            case PM_Q1: case PM_REF2: w = c1[oc]; break;
            case PM_Q2: case PM_REF3: w = c2[oc]; break;
            case PM_PRJ2:
                if (cst[k] == 1) w = g.rk == 2 ? T(2) * ce[oc] - c0[oc] : T(4) * c2[oc] - T(3) * c0[oc];
                else w = T(2) * c1[oc] - c0[oc];
                break;
            case PM_PRJ3: w = ce[oc]; break;
            default: w = c0[oc]; break; // PM_MID: children at t^n
            }
            acc += w;
        }
        const T mean = acc * T(1.0 / NCH);
        switch (mode) {
        case PM_Q0: q0[o] = mean; break;
        case PM_Q1: case PM_PRJ2: q1[o] = mean; break;
        case PM_Q2: q2[o] = mean; break;
        case PM_REF2:
            nd<T>(g, F_XH, sl)[o] = mean;
            q1[o] = T(2) * mean - q0[o];
            break;
        case PM_REF3: {
            nd<T>(g, F_N1, sl)[o] = mean;
            nd<T>(g, F_N3, sl)[o] = T(-6.5) * q0[o] - T(1.5) * q1[o] + T(9) * mean;
            q2[o] = T(-5.5) * q0[o] - T(1.5) * q1[o] + T(8) * mean;
            break;
        }
        case PM_PRJ3:
            q2[o] = mean;
            qe[o] = T(2) * mean - q0[o];
            break;
        default: { // PM_MID
            if (g.rk == 2) {
                nd<T>(g, F_NH, sl)[o] = mean;
                qe[o] = T(-2) * q0[o] - q1[o] + T(4) * mean;
            } else {
                q2[o] = mean;
                qe[o] = T(2) * mean - q0[o];
                const T n1 = (mean + T(5.5) * q0[o] + T(1.5) * q1[o]) * T(0.125);
                nd<T>(g, F_N1, sl)[o] = n1;
                nd<T>(g, F_N3, sl)[o] = T(-6.5) * q0[o] - T(1.5) * q1[o] + T(9) * n1;
            }
        }
        }
    }
}

template <int D, class T>
__device__ __forceinline__ void dev_project(const Grid& g, int l, int mode)
{
    const int cnt = g.counts[LMAX + 1 + l];
    const int* list = g.inner + g.off[l];
    const long long N = g.N[l];
    MRLT_GRID_STRIDE(t, cnt)
    {
        const long long id = list[t];
        if (id < 0 || id >= N) {
            atomicOr(g.err, ERR_INDEX);
            continue;
        }
        project_node<D, T>(g, l, id, mode);
    }
}

// An up-sweep of one mode over levels hi..lo (hi - lo = depth >= 1) in one
// launch.  Each step of a CTA takes `tops` internal nodes of level lo and
// projects their internal descendants bottom-up, level by level, with a CTA
// barrier between levels: a node's projection reads only its own children,
// which lie in the same subtree.  Thread t of a step owns descendant t % sub
// of top node t / sub on each level (sub = 2^{d (m - lo)} on level m), so
// 2^{d depth} <= blockDim.x is required.  Every node is projected by the same
// operations as in dev_project.
template <int D, class T>
__device__ __forceinline__ void dev_project_up(const Grid& g, int hi, int lo, int mode)
{
    const int depth = hi - lo;
    const int tops = blockDim.x >> (D * depth);
    const int cnt = g.counts[LMAX + 1 + lo];
    const int* list = g.inner + g.off[lo];
    const long long N = g.N[lo];
    const int nstep = (cnt + tops - 1) / tops;
    for (int c = blockIdx.x; c < nstep; c += gridDim.x) { // uniform across the CTA
        for (int m = hi; m >= lo; --m) {
            const int s = m - lo;
            const int sub = 1 << (D * s);
            const int t = threadIdx.x;
            const int ti = c * tops + t / sub;
            if (t < tops * sub && ti < cnt) {
                const long long top = list[ti];
                if (top < 0 || top >= N) {
                    atomicOr(g.err, ERR_INDEX);
                } else {
                    int tc[3];
                    cell_xyz(g, lo, top, tc);
                    const int r = t % sub, msk = (1 << s) - 1;
                    const long long id = cell_id(g, m, (tc[0] << s) + (r & msk),
                                                 D > 1 ? (tc[1] << s) + ((r >> s) & msk) : 0,
                                                 D > 2 ? (tc[2] << s) + (r >> (2 * s)) : 0);
                    if (status(g, m, id) == 2) project_node<D, T>(g, m, id, mode);
                }
            }
            __syncthreads();
        }
    }
}

// ------------------------------------------------------------ adaptation
__device__ __forceinline__ double eps_level(const Grid& g, int l)
{
    return g.eps_mode == 1 ? ldexp(g.eps, g.d * (l - g.L)) : g.eps;
}

// detail norm (Eq. 5) of every internal node of levels lo..hi (< L): max over
// children and variables of |q_child - prediction| / s_v; flags significance
// (> eps_{l+1}) and the scale-safety bound (> 8 eps_{l+1}).  The predictions
// and the test are FP64 whatever the storage type T.
template <int D, int M, class T>
__device__ __forceinline__ void dev_detail(const Grid& g, int lo, int hi)
{
    double sc[M];
#pragma unroll
    for (int v = 0; v < M; ++v) sc[v] = __longlong_as_double((long long)g.scale_bits[v]);
    for (int l = lo; l <= hi; ++l) {
        const int cnt = g.counts[LMAX + 1 + l];
        const int* list = g.inner + g.off[l];
        const long long N = g.N[l];
        const double el = eps_level(g, l + 1);
        MRLT_GRID_STRIDE(t, cnt)
        {
            const long long id = list[t];
            if (id < 0 || id >= N) {
                atomicOr(g.err, ERR_INDEX);
                continue;
            }
            uint8_t fl = 0;
            if (g.eps <= 0.0) {
                fl = FL_SIG;
            } else {
                int c[3];
                cell_xyz(g, l, id, c);
                const Ctx x{l, 0, g.lb};
                double nrm = 0.0;
                double p[1 << D][M];
                predict_children<D, M, T>(g, x, l, c, p);
#pragma unroll
                for (int k = 0; k < (1 << D); ++k) {
                    const long long cid = cell_id(g, l + 1, 2 * c[0] + (k & 1), D > 1 ? 2 * c[1] + ((k >> 1) & 1) : 0,
                                                  D > 2 ? 2 * c[2] + ((k >> 2) & 1) : 0);
                    const T* qc = nd<T>(g, F_Q0, slot_of(g, l + 1, cid));
#pragma unroll
                    for (int v = 0; v < M; ++v) nrm = fmax(nrm, fabs(double(qc[v]) - p[k][v]) / sc[v]);
                }
                if (fabs(nrm - el) <= 1e-10 * el || fabs(nrm - 8.0 * el) <= 8e-10 * el)
                    atomicAdd(g.near, 1ull);
                if (nrm > el) fl |= FL_SIG;
                if (nrm > 8.0 * el) fl |= FL_BIG;
            }
            g.flag[g.off[l] + id] |= fl;
        }
    }
}

template <int D>
__device__ __forceinline__ bool nb3(const Grid& g, int l, const int c[3], int dx, int dy, int dz, long long* id)
{
    int q[3] = {0, 0, 0};
    if (!in_box(g, l, 0, c[0] + dx, &q[0])) return false;
    if (D > 1 && !in_box(g, l, 1, c[1] + dy, &q[1])) return false;
    if (D > 2 && !in_box(g, l, 2, c[2] + dz, &q[2])) return false;
    *id = cell_id(g, l, q[0], q[1], q[2]);
    return true;
}

#define MRLT_FOR3(D, dx, dy, dz)                                  \
    for (int dz = (D > 2 ? -1 : 0); dz <= (D > 2 ? 1 : 0); ++dz) \
        for (int dy = (D > 1 ? -1 : 0); dy <= (D > 1 ? 1 : 0); ++dy) \
            for (int dx = -1; dx <= 1; ++dx)

// desired refinement of levels lo..hi: significant node in the 3^d
// neighbourhood (space safety), or parent flagged by scale safety (parent
// level >= la); eps = 0 refines all
template <int D>
__device__ __forceinline__ void dev_desire(const Grid& g, int lo, int hi, int la)
{
    for (int l = lo; l <= hi; ++l) {
        const long long N = g.N[l];
        uint8_t* fl = g.flag + g.off[l];
        MRLT_GRID_STRIDE(id, N)
        {
            bool want = g.eps <= 0.0;
            if (!want) {
                int c[3];
                cell_xyz(g, l, id, c);
                MRLT_FOR3(D, dx, dy, dz)
                {
                    long long j;
                    if (nb3<D>(g, l, c, dx, dy, dz, &j) && (fl[j] & FL_SIG)) want = true;
                }
                if (!want && l - 1 >= la) {
                    const long long p = cell_id(g, l - 1, c[0] >> 1, c[1] >> 1, c[2] >> 1);
                    if (g.flag[g.off[l - 1] + p] & FL_BIG) want = true;
                }
            }
            if (want) fl[id] |= FL_DES;
        }
    }
}

// Admissible refinements of levels lo..hi and R = desired and admissible.
// A node (l, i) may be refined if every node of the frozen level la-1 its
// grading chain requires is refined already.  Unrolling the rule "refining
// (m, j) needs (m-1, floor(j/2) + delta), |delta| <= 1" from level l down to
// la-1 gives, per direction, the interval [a, b] obtained by
// a -> floor(a/2) - 1, b -> floor(b/2) + 1 (l - la + 1 times), wrapped when
// periodic and clipped at walls.  At a full adaptation (la = min level)
// everything is admissible.
template <int D>
__device__ __forceinline__ void dev_allow(const Grid& g, int lo, int hi, int la)
{
    for (int l = lo; l <= hi; ++l) {
        const long long N = g.N[l];
        uint8_t* fl = g.flag + g.off[l];
        MRLT_GRID_STRIDE(id, N)
        {
            bool ok = true;
            if (la > g.lb) {
                int c[3];
                cell_xyz(g, l, id, c);
                const int pl = la - 1, n = g.n[pl];
                int lo3[3] = {0, 0, 0}, cnt3[3] = {1, 1, 1};
                for (int k = 0; k < D; ++k) {
                    int a = c[k], b = c[k];
                    for (int m = l; m >= la; --m) {
                        a = (a >> 1) - 1; // arithmetic shift: floor for negatives
                        b = (b >> 1) + 1;
                    }
                    if (g.bc[k] == 0) {
                        lo3[k] = a;
                        cnt3[k] = min(b - a + 1, n);
                    } else {
                        lo3[k] = max(a, 0);
                        cnt3[k] = min(b, n - 1) - lo3[k] + 1;
                    }
                }
                for (int tz = 0; tz < cnt3[2] && ok; ++tz)
                    for (int ty = 0; ty < cnt3[1] && ok; ++ty)
                        for (int tx = 0; tx < cnt3[0] && ok; ++tx) {
                            int q[3] = {lo3[0] + tx, lo3[1] + ty, lo3[2] + tz};
                            for (int k = 0; k < D; ++k)
                                if (g.bc[k] == 0) q[k] &= n - 1; // periodic wrap (n = 2^l)
                            ok = status(g, pl, cell_id(g, pl, q[0], q[1], q[2])) == 2;
                        }
            }
            uint8_t f = fl[id];
            if (ok) {
                f |= FL_ALLOW;
                if (f & FL_DES) f |= FL_REF;
            }
            fl[id] = f;
        }
    }
}

// grading closure, one level: refining (l, i) refines (l-1, floor(i/2) + delta)
// for |delta|_inf <= 1 -- gathered at the coarse node
template <int D>
__device__ __forceinline__ void dev_close(const Grid& g, int l)
{
    const int pl = l - 1;
    const long long N = g.N[pl];
    uint8_t* fp = g.flag + g.off[pl];
    const uint8_t* fc = g.flag + g.off[l];
    MRLT_GRID_STRIDE(pid, N)
    {
        if (fp[pid] & FL_REF) continue;
        int c[3];
        cell_xyz(g, pl, pid, c);
        bool hit = false;
        MRLT_FOR3(D, dx, dy, dz)
        {
            long long j;
            if (!nb3<D>(g, pl, c, -dx, -dy, -dz, &j)) continue;
            int q[3];
            cell_xyz(g, pl, j, q);
            for (int k = 0; k < (1 << D); ++k) {
                const long long cid = cell_id(g, l, 2 * q[0] + (k & 1), D > 1 ? 2 * q[1] + ((k >> 1) & 1) : 0,
                                              D > 2 ? 2 * q[2] + ((k >> 2) & 1) : 0);
                if (fc[cid] & FL_REF) hit = true;
            }
        }
        if (hit) fp[pid] |= FL_REF;
    }
}

// Does the tree flagged by a remesh at level la (fine iteration it) fit the
// node arrays?  Each thread of the kernel that finalises the flags counted
// `c` refined cells (the kernel's cells of levels la..L-1 in one flat
// grid-stride range over them); the blocks add their counts into room[0].
// The new tree has 2^d nodes above level la per refined cell, and the slots
// it may take are the free ones plus those of the nodes above level la now
// (the remesh releases them first).  The last block to finish (ticket
// room[3]) decides: short of slots, the solver halts at this iteration,
// room[1] = it + 1, room[2] = the nodes of the new tree (see halted()).
// Called by every thread of the block.
__device__ __forceinline__ void room_decide(const Grid& g, int c, int la, long long it)
{
    __shared__ int blk;
    if (threadIdx.x == 0) blk = 0;
    __syncthreads();
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(&blk, c);
    __syncthreads();
    if (threadIdx.x != 0) return;
    if (blk) atomicAdd(&g.room[0], blk);
    __threadfence();
    if (atomicAdd(&g.room[3], 1) != (int)gridDim.x - 1) return;
    __threadfence();
    const long long fresh = (long long)atomicExch(&g.room[0], 0) << g.d;
    g.room[3] = 0;
    long long above = 0, below = 0;
    for (int l = g.lb; l <= g.L; ++l) {
        const long long n = (long long)g.counts[l] + g.counts[LMAX + 1 + l];
        if (l > la) above += n;
        else below += n;
    }
    if (fresh > g.ftop[0] + above) {
        g.room[2] = (int)(below + fresh);
        g.room[1] = (int)(it + 1);
    }
}

// refined cells among this thread's cells of the flat range [off[la], off[L])
// (levels la..L-1), in the grid-stride order of the kernel's own pass
__device__ __forceinline__ int refined_here(const Grid& g, int la)
{
    int c = 0;
    const long long from = g.off[la];
    MRLT_GRID_STRIDE(i, g.off[g.L] - from) c += (g.flag[from + i] & FL_REF) ? 1 : 0;
    return c;
}

// Slots of the nodes a remesh removes (levels la+1..L: a node whose parent
// is not refined any more), pushed on the free stack before the apply passes
// pop slots for new nodes.  Walks the node lists of the tree being replaced.
static __device__ __forceinline__ void dev_release(const Grid& g, int la)
{
    for (int l = la + 1; l <= g.L; ++l) {
        const long long N = g.N[l];
        for (int which = 0; which < 2; ++which) {
            const int cnt = g.counts[which * (LMAX + 1) + l];
            const int* list = (which ? g.inner : g.leaves) + g.off[l];
            MRLT_GRID_STRIDE(t, cnt)
            {
                const long long id = list[t];
                if (id < 0 || id >= N) {
                    atomicOr(g.err, ERR_INDEX);
                    continue;
                }
                int c[3];
                cell_xyz(g, l, id, c);
                const long long p = cell_id(g, l - 1, c[0] >> 1, c[1] >> 1, c[2] >> 1);
                if (g.flag[g.off[l - 1] + p] & FL_REF) continue; // stays
                const int sl = slot_of(g, l, id);
                if (sl > 0) g.fstack[atomicAdd(&g.ftop[0], 1)] = sl;
                g.slot[g.off[l] + id] = -1;
            }
        }
    }
}

// install the new tree on level l (top-down): status from the refinement
// flags; new nodes take a free slot (the sink, with ERR_CAPACITY, when none
// is left) and are predicted from level l-1 (Sec. 2, in FP64, stored as T);
// new leaves and merged nodes get q^{n+1} = q^n; registers of changed nodes
// cleared
template <int D, int M, class T>
__device__ __forceinline__ void dev_apply(const Grid& g, int l, int la)
{
    const long long N = g.N[l];
    const int top = g.ftop[0]; // free slots after this remesh's releases
    MRLT_GRID_STRIDE(id, N)
    {
        const uint8_t old = status(g, l, id);
        int c[3];
        cell_xyz(g, l, id, c);
        bool exists;
        if (l == la) exists = old != 0;
        else {
            const long long p = cell_id(g, l - 1, c[0] >> 1, c[1] >> 1, c[2] >> 1);
            exists = (g.flag[g.off[l - 1] + p] & FL_REF) != 0;
        }
        const bool refined = l < g.L && (g.flag[g.off[l] + id] & FL_REF);
        if (refined && !exists) atomicOr(g.err, ERR_SOURCE);
        const uint8_t nw = exists ? (refined ? 2 : 1) : 0;
        if (nw == old) continue;
        g.st[g.off[l] + id] = nw;
        if (nw == 0) continue; // removed: its slot was released before the apply passes
        int sl;
        if (old == 0) {
            const int k = atomicAdd(&g.ftop[1], 1);
            sl = k < top ? g.fstack[top - 1 - k] : 0;
            if (k >= top) atomicOr(g.err, ERR_CAPACITY);
            g.slot[g.off[l] + id] = sl;
        } else {
            sl = slot_of(g, l, id);
        }
        T* q0 = nd<T>(g, F_Q0, sl);
        if (old == 0) {
            const Ctx x{l, 0, g.lb};
            double p[M];
            predict<D, M, T, double>(g, x, l, c, p);
#pragma unroll
            for (int v = 0; v < M; ++v) q0[v] = T(p[v]);
        }
        if (nw == 1) {
            T* qe = nd<T>(g, F_QE, sl);
#pragma unroll
            for (int v = 0; v < M; ++v) qe[v] = q0[v];
        }
        if (g.rg) {
            double* rg = regs(g.rg, g, sl);
            for (int r = 0; r < g.nf * M; ++r) rg[r] = 0.0;
        }
    }
}

// adaptation flags of levels >= la cleared (grid-stride)
static __device__ __forceinline__ void dev_clear_flags(const Grid& g, long long from, long long to)
{
    MRLT_GRID_STRIDE(i, to - from) g.flag[from + i] = 0;
}

// ------------------------------------------------------------ compaction
// Chunks of CH consecutive cells of one level, numbered over levels lo..hi:
// level l owns the chunks [base[l], base[l+1]).
struct LevelChunks {
    int lo, hi;
    int base[LMAX + 2];
};

__device__ __forceinline__ int chunk_level(const LevelChunks& b, int c)
{
    int l = b.lo;
    while (l < b.hi && c >= b.base[l + 1]) ++l;
    return l;
}

// Per chunk (a CTA of CH threads, one cell each): number of leaves and of
// internal nodes, into bc[2 chunk], bc[2 chunk + 1].
template <int CH>
__device__ __forceinline__ void chunk_count(const Grid& g, const LevelChunks& lc, int chunk, int* bc)
{
    __shared__ int wl[CH / 32], wi[CH / 32];
    const int l = chunk_level(lc, chunk);
    const long long N = g.N[l];
    const long long i = (long long)(chunk - lc.base[l]) * CH + threadIdx.x;
    const int s = i < N ? status(g, l, i) : 0;
    if (i < N) g.flag[g.off[l] + i] = 0; // the remesh is installed: its flags are spent
    const unsigned bl = __ballot_sync(0xffffffffu, s == 1);
    const unsigned bi = __ballot_sync(0xffffffffu, s == 2);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        wl[warp] = __popc(bl);
        wi[warp] = __popc(bi);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int a = 0, b = 0;
        for (int w = 0; w < CH / 32; ++w) {
            a += wl[w];
            b += wi[w];
        }
        bc[2 * chunk] = a;
        bc[2 * chunk + 1] = b;
        if (chunk == 0) { // the slots popped by the remesh leave the free stack
            const int k = g.ftop[1], top = g.ftop[0];
            g.ftop[0] = top - (k < top ? k : top);
            g.ftop[1] = 0;
        }
    }
    __syncthreads();
}

// Exclusive scan of the chunk counts of level l by one CTA of NT threads;
// level totals to counts[l], counts[LMAX + 1 + l].
template <int NT>
__device__ __forceinline__ void level_scan(const Grid& g, const LevelChunks& lc, int l, int* bc)
{
    __shared__ int sa[NT], sb[NT];
    const int b0l = lc.base[l], nb = lc.base[l + 1] - b0l;
    const int tid = threadIdx.x;
    const int per = (nb + NT - 1) / NT;
    const int b0 = b0l + tid * per, b1 = min(b0 + per, b0l + nb);
    int a = 0, b = 0;
    for (int i = b0; i < b1; ++i) {
        a += bc[2 * i];
        b += bc[2 * i + 1];
    }
    sa[tid] = a;
    sb[tid] = b;
    __syncthreads();
    for (int o = 1; o < NT; o <<= 1) {
        const int xa = tid >= o ? sa[tid - o] : 0;
        const int xb = tid >= o ? sb[tid - o] : 0;
        __syncthreads();
        sa[tid] += xa;
        sb[tid] += xb;
        __syncthreads();
    }
    int ea = sa[tid] - a, eb = sb[tid] - b;
    for (int i = b0; i < b1; ++i) {
        const int ta = bc[2 * i], tb = bc[2 * i + 1];
        bc[2 * i] = ea;
        bc[2 * i + 1] = eb;
        ea += ta;
        eb += tb;
    }
    if (tid == NT - 1) {
        g.counts[l] = sa[NT - 1];
        g.counts[LMAX + 1 + l] = sb[NT - 1];
    }
    __syncthreads();
}

// the leaf's tile of the tiled stage kernel is active
__device__ __forceinline__ void mark_tile(const Grid& g, int l, long long i)
{
    const int tx = g.d == 1 ? kTile1X : (g.d == 2 ? kTile2X : kTile3X);
    const int ty = g.d == 2 ? kTile2Y : kTile3Y;
    const long long mask = (1LL << l) - 1;
    const long long x = i & mask, y = g.d >= 2 ? (i >> l) & mask : 0, z = g.d == 3 ? i >> (2 * l) : 0;
    g.tflag[g.toff[l] + x / tx + (long long)g.ntx[l] * (y / ty + (long long)g.nty[l] * (z / kTile3Z))] = 1;
}

// Per chunk: leaves and internal nodes written to the level lists at the
// scanned offsets (ascending cell id), tiles holding a leaf flagged.
template <int CH>
__device__ __forceinline__ void chunk_scatter(const Grid& g, const LevelChunks& lc, int chunk, const int* bc)
{
    __shared__ int wl[CH / 32], wi[CH / 32];
    const int l = chunk_level(lc, chunk);
    const long long N = g.N[l];
    const long long i = (long long)(chunk - lc.base[l]) * CH + threadIdx.x;
    const int s = i < N ? status(g, l, i) : 0;
    const unsigned bl = __ballot_sync(0xffffffffu, s == 1);
    const unsigned bi = __ballot_sync(0xffffffffu, s == 2);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        wl[warp] = __popc(bl);
        wi[warp] = __popc(bi);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int a = bc[2 * chunk], b = bc[2 * chunk + 1];
        for (int w = 0; w < CH / 32; ++w) {
            const int ta = wl[w], tb = wi[w];
            wl[w] = a;
            wi[w] = b;
            a += ta;
            b += tb;
        }
    }
    __syncthreads();
    const unsigned below = (1u << lane) - 1u;
    if (s == 1) g.leaves[g.off[l] + wl[warp] + __popc(bl & below)] = (int)i;
    if (s == 2) g.inner[g.off[l] + wi[warp] + __popc(bi & below)] = (int)i;
    if (s == 1) mark_tile(g, l, i);
    __syncthreads();
}

// ordered list of the active tiles of level l by one CTA of NT threads
template <int NT>
__device__ __forceinline__ void level_tile_list(const Grid& g, int l)
{
    __shared__ int sc[NT];
    const int nt = g.ntx[l] * g.nty[l] * g.ntz[l];
    const uint8_t* fl = g.tflag + g.toff[l];
    const int tid = threadIdx.x, per = (nt + NT - 1) / NT;
    const int t0 = tid * per, t1 = min(t0 + per, nt);
    int c = 0;
    for (int t = t0; t < t1; ++t) c += fl[t] != 0;
    sc[tid] = c;
    __syncthreads();
    for (int o = 1; o < NT; o <<= 1) {
        const int xo = tid >= o ? sc[tid - o] : 0;
        __syncthreads();
        sc[tid] += xo;
        __syncthreads();
    }
    int pos = sc[tid] - c;
    for (int t = t0; t < t1; ++t)
        if (fl[t]) g.tlist[g.toff[l] + pos++] = t;
    if (tid == NT - 1) g.counts[2 * (LMAX + 1) + l] = sc[NT - 1];
    __syncthreads();
}

// ------------------------------------------------------------ registers
// conservative correction of the coarse leaves of level l whose step ended:
// q += +-(coarse time-integrated flux - mean of the fine ones) / dx; the
// registers read are cleared for the next step
template <int D, class T>
__device__ __forceinline__ void dev_reflux(const Grid& g, int lo, int hi)
{
    for (int l = lo; l <= hi; ++l) {
        const int cnt = g.counts[l];
        const int* list = g.leaves + g.off[l];
        const long long N = g.N[l];
        const int m = g.m;
        constexpr int NT = 1 << (D - 1);
        MRLT_GRID_STRIDE(t, cnt)
        {
            const long long id = list[t];
            if (id < 0 || id >= N) {
                atomicOr(g.err, ERR_INDEX);
                continue;
            }
            int c[3];
            cell_xyz(g, l, id, c);
            for (int fi = 0; fi < 2 * D; ++fi) {
                const int k = fi >> 1, side = (fi & 1) ? 1 : -1;
                int q;
                if (!in_box(g, l, k, c[k] + side, &q)) continue;
                int nb[3] = {c[0], c[1], c[2]};
                nb[k] = q;
                if (status(g, l, cell_id(g, l, nb[0], nb[1], nb[2])) != 2) continue;
                const int opp = 2 * k + (side > 0 ? 0 : 1);
                long long ch[NT];
                for (int tt = 0; tt < NT; ++tt) {
                    int p[3] = {0, 0, 0}, bit = 0;
                    for (int j = 0; j < D; ++j) {
                        if (j == k) continue;
                        p[j] = 2 * nb[j] + ((tt >> bit) & 1);
                        ++bit;
                    }
                    p[k] = 2 * nb[k] + (side > 0 ? 0 : 1);
                    ch[tt] = cell_id(g, l + 1, p[0], p[1], p[2]);
                    if (status(g, l + 1, ch[tt]) != 1) atomicOr(g.err, ERR_REFLUX);
                }
                const int sl = slot_of(g, l, id);
                double* rc = regs(g.rg, g, sl);
                int csl[NT];
                for (int tt = 0; tt < NT; ++tt) csl[tt] = slot_of(g, l + 1, ch[tt]);
                T* qe = nd<T>(g, F_QE, sl);
                const double idx = 1.0 / g.dx[l][k];
                for (int v = 0; v < m; ++v) {
                    double sum = 0.0;
                    for (int tt = 0; tt < NT; ++tt) {
                        double* r = regs(g.rg, g, csl[tt]) + opp * m + v;
                        sum += *r;
                        *r = 0.0;
                    }
                    double* r = rc + fi * m + v;
                    // the correction from the FP64 registers, rounded to T once
                    qe[v] = T(double(qe[v]) + side * (*r - sum * (1.0 / NT)) * idx);
                    *r = 0.0;
                }
            }
        }
    }
}

// ------------------------------------------------------------ reductions
// running max |q^n_v| over the leaves of levels lo..hi (detail normalisation)
template <class T>
__device__ __forceinline__ void dev_scale(const Grid& g, int lo, int hi)
{
    for (int l = lo; l <= hi; ++l) {
        const int cnt = g.counts[l];
        const int* list = g.leaves + g.off[l];
        const long long N = g.N[l];
        double mx[MMAX] = {0.0, 0.0, 0.0, 0.0, 0.0};
        MRLT_GRID_STRIDE(t, cnt)
        {
            const long long id = list[t];
            if (id < 0 || id >= N) continue;
            const T* q0 = nd<T>(g, F_Q0, slot_of(g, l, id));
            for (int v = 0; v < g.m; ++v) mx[v] = fmax(mx[v], fabs(double(q0[v])));
        }
        for (int v = 0; v < g.m; ++v) {
            double a = mx[v];
            for (int o = 16; o > 0; o >>= 1) a = fmax(a, __shfl_xor_sync(0xffffffffu, a, o));
            if ((threadIdx.x & 31) == 0 && a > 0.0)
                atomicMax(&g.scale_bits[v], (unsigned long long)__double_as_longlong(a));
        }
    }
}

// non-finite end values of the leaves of levels lo..hi set ERR_NONFINITE
template <class T>
__device__ __forceinline__ void dev_finite(const Grid& g, int lo, int hi)
{
    for (int l = lo; l <= hi; ++l) {
        const int cnt = g.counts[l];
        const int* list = g.leaves + g.off[l];
        const long long N = g.N[l];
        MRLT_GRID_STRIDE(t, cnt)
        {
            const long long id = list[t];
            if (id < 0 || id >= N) continue;
            const T* qe = nd<T>(g, F_QE, slot_of(g, l, id));
            for (int v = 0; v < g.m; ++v)
                if (!isfinite(double(qe[v]))) atomicOr(g.err, ERR_NONFINITE);
        }
    }
}

// largest sum of characteristic speeds over the leaves of levels lo..hi (CFL
// step), as the bit pattern of a positive double in *g.wmax
template <int EQ, int D, class T>
__device__ __forceinline__ void dev_wave(const Grid& g, int lo, int hi)
{
    constexpr int M = EQ == 2 ? D + 2 : 1;
    double w = 0.0;
    for (int l = lo; l <= hi; ++l) {
        const int cnt = g.counts[l];
        const int* list = g.leaves + g.off[l];
        const long long N = g.N[l];
        MRLT_GRID_STRIDE(t, cnt)
        {
            const long long id = list[t];
            if (id < 0 || id >= N) continue;
            const T* qe = nd<T>(g, F_QE, slot_of(g, l, id));
            double q[M];
#pragma unroll
            for (int v = 0; v < M; ++v) q[v] = double(qe[v]);
            const double s = wave_speed<EQ, D, M>(g, q);
            w = fmax(w, s != s ? 1e300 : s);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w = fmax(w, __shfl_xor_sync(0xffffffffu, w, o));
    if ((threadIdx.x & 31) == 0 && w > 0.0) atomicMax(g.wmax, (unsigned long long)__double_as_longlong(w));
}

} // namespace mrlt

// mrlt_tree.cu -- tree kernels of the MRLT library: projections and tree
// refreshing (Eqs. 3, 15-22; Algs. 3, 4, 6, 8, 9), the multiresolution
// adaptation (details Eq. 5, thresholding Alg. 2, graded closure Alg. 1),
// warp-ballot compaction of the per-level leaf / internal-node lists,
// conservative flux registers, reductions and read-back packing.
#include "mrlt_tree.cuh"

namespace mrlt {

static inline int blocks_dense(long long n)
{
    long long b = (n + NTHREADS - 1) / NTHREADS;
    return (int)(b < 1 ? 1 : (b > 65535 ? 65535 : b));
}
static inline int blocks_list(const Grid& g, int l)
{
    long long b = (g.N[l] + NTHREADS - 1) / NTHREADS;
    return (int)(b < 1 ? 1 : (b > 1216 ? 1216 : b));
}

#define GRID_STRIDE(i, n) \
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < (n); i += (long long)gridDim.x * blockDim.x)

// ------------------------------------------------------------ simple leaf copies
__global__ void k_leaf_copy(Grid g, int lo, int hi, int from, int to)
{
    pdl_enter();
    for (int l = lo; l <= hi; ++l) {
        const int cnt = g.counts[l];
        const int* list = g.leaves + g.off[l];
        const long long N = g.N[l];
        const double* a = fbase(g, from, l);
        double* b = fbase_w(g, to, l);
        GRID_STRIDE(t, cnt)
        {
            const long long id = list[t];
            if (id < 0 || id >= N) {
                atomicOr(g.err, ERR_INDEX);
                continue;
            }
            for (int v = 0; v < g.m; ++v) b[v * N + id] = a[v * N + id];
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
template <int D>
__global__ void k_project(Grid g, int l, int mode)
{
    pdl_enter();
    const int cnt = g.counts[LMAX + 1 + l];
    const int* list = g.inner + g.off[l];
    const long long N = g.N[l], Nc = g.N[l + 1];
    constexpr int NCH = 1 << D;
    GRID_STRIDE(t, cnt)
    {
        const long long id = list[t];
        if (id < 0 || id >= N) {
            atomicOr(g.err, ERR_INDEX);
            continue;
        }
        int c[3];
        cell_xyz(g, l, id, c);
        long long ch[NCH];
        uint8_t cst[NCH];
#pragma unroll
        for (int k = 0; k < NCH; ++k) {
            ch[k] = cell_id(g, l + 1, 2 * c[0] + (k & 1), D > 1 ? 2 * c[1] + ((k >> 1) & 1) : 0,
                            D > 2 ? 2 * c[2] + ((k >> 2) & 1) : 0);
            cst[k] = status(g, l + 1, ch[k]);
        }
        const double* c0 = fbase(g, F_Q0, l + 1);
        const double* c1 = fbase(g, F_Q1, l + 1);
        const double* c2 = fbase(g, F_Q2, l + 1);
        const double* ce = fbase(g, F_QE, l + 1);
        double* q0 = fbase_w(g, F_Q0, l);
        double* q1 = fbase_w(g, F_Q1, l);
        double* q2 = fbase_w(g, F_Q2, l);
        double* qe = fbase_w(g, F_QE, l);
        for (int v = 0; v < g.m; ++v) {
            const long long o = v * N + id;
            double acc = 0.0;
#pragma unroll
            for (int k = 0; k < NCH; ++k) {
                const long long oc = v * Nc + ch[k];
                double w;
                switch (mode) {
                case PM_Q0: w = c0[oc]; break;
                case PM_Q1: case PM_REF2: w = c1[oc]; break;
                case PM_Q2: case PM_REF3: w = c2[oc]; break;
                case PM_PRJ2:
                    if (cst[k] == 1) w = g.rk == 2 ? 2.0 * ce[oc] - c0[oc] : 4.0 * c2[oc] - 3.0 * c0[oc];
                    else w = 2.0 * c1[oc] - c0[oc];
                    break;
                case PM_PRJ3: w = ce[oc]; break;
                default: w = c0[oc]; break; // PM_MID: children at t^n
                }
                acc += w;
            }
            const double mean = acc * (1.0 / NCH);
            switch (mode) {
            case PM_Q0: q0[o] = mean; break;
            case PM_Q1: case PM_PRJ2: q1[o] = mean; break;
            case PM_Q2: q2[o] = mean; break;
            case PM_REF2:
                fbase_w(g, F_XH, l)[o] = mean;
                q1[o] = 2.0 * mean - q0[o];
                break;
            case PM_REF3: {
                fbase_w(g, F_N1, l)[o] = mean;
                fbase_w(g, F_N3, l)[o] = -6.5 * q0[o] - 1.5 * q1[o] + 9.0 * mean;
                q2[o] = -5.5 * q0[o] - 1.5 * q1[o] + 8.0 * mean;
                break;
            }
            case PM_PRJ3:
                q2[o] = mean;
                qe[o] = 2.0 * mean - q0[o];
                break;
            default: { // PM_MID
                if (g.rk == 2) {
                    fbase_w(g, F_NH, l)[o] = mean;
                    qe[o] = -2.0 * q0[o] - q1[o] + 4.0 * mean;
                } else {
                    q2[o] = mean;
                    qe[o] = 2.0 * mean - q0[o];
                    const double n1 = (mean + 5.5 * q0[o] + 1.5 * q1[o]) * 0.125;
                    fbase_w(g, F_N1, l)[o] = n1;
                    fbase_w(g, F_N3, l)[o] = -6.5 * q0[o] - 1.5 * q1[o] + 9.0 * n1;
                }
            }
            }
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
// (> eps_{l+1}) and the scale-safety bound (> 8 eps_{l+1})
template <int D, int M>
__global__ void k_detail(Grid g, int lo, int hi)
{
    pdl_enter();
    double sc[M];
#pragma unroll
    for (int v = 0; v < M; ++v) sc[v] = __longlong_as_double((long long)g.scale_bits[v]);
    for (int l = lo; l <= hi; ++l) {
        const int cnt = g.counts[LMAX + 1 + l];
        const int* list = g.inner + g.off[l];
        const long long N = g.N[l], Nc = g.N[l + 1];
        const double el = eps_level(g, l + 1);
        GRID_STRIDE(t, cnt)
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
#pragma unroll 1
                for (int k = 0; k < (1 << D); ++k) {
                    int q[3] = {2 * c[0] + (k & 1), D > 1 ? 2 * c[1] + ((k >> 1) & 1) : 0,
                                D > 2 ? 2 * c[2] + ((k >> 2) & 1) : 0};
                    double p[M];
                    predict<D, M>(g, x, l + 1, q, p);
                    const long long cid = cell_id(g, l + 1, q[0], q[1], q[2]);
                    const double* qc = fbase(g, F_Q0, l + 1) + cid;
#pragma unroll
                    for (int v = 0; v < M; ++v) nrm = fmax(nrm, fabs(qc[v * Nc] - p[v]) / sc[v]);
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

#define FOR3(D, dx, dy, dz)                                       \
    for (int dz = (D > 2 ? -1 : 0); dz <= (D > 2 ? 1 : 0); ++dz) \
        for (int dy = (D > 1 ? -1 : 0); dy <= (D > 1 ? 1 : 0); ++dy) \
            for (int dx = -1; dx <= 1; ++dx)

// desired refinement of levels lo..hi: significant node in the 3^d
// neighbourhood (space safety), or parent flagged by scale safety (parent
// level >= la); eps = 0 refines all
template <int D>
__global__ void k_desire(Grid g, int lo, int hi, int la)
{
    pdl_enter();
    for (int l = lo; l <= hi; ++l) {
        const long long N = g.N[l];
        uint8_t* fl = g.flag + g.off[l];
        GRID_STRIDE(id, N)
        {
            bool want = g.eps <= 0.0;
            if (!want) {
                int c[3];
                cell_xyz(g, l, id, c);
                FOR3(D, dx, dy, dz)
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
__global__ void k_allow(Grid g, int lo, int hi, int la)
{
    pdl_enter();
    for (int l = lo; l <= hi; ++l) {
        const long long N = g.N[l];
        uint8_t* fl = g.flag + g.off[l];
        GRID_STRIDE(id, N)
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
                                if (g.bc[k] == 0) q[k] = ((q[k] % n) + n) % n;
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
__global__ void k_close(Grid g, int l)
{
    pdl_enter();
    const int pl = l - 1;
    const long long N = g.N[pl];
    uint8_t* fp = g.flag + g.off[pl];
    const uint8_t* fc = g.flag + g.off[l];
    GRID_STRIDE(pid, N)
    {
        if (fp[pid] & FL_REF) continue;
        int c[3];
        cell_xyz(g, pl, pid, c);
        bool hit = false;
        FOR3(D, dx, dy, dz)
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

// install the new tree on level l (top-down): status from the refinement
// flags; new nodes predicted from level l-1 (Sec. 2); new leaves and merged
// nodes get q^{n+1} = q^n; registers of changed nodes cleared
template <int D, int M>
__global__ void k_apply(Grid g, int l, int la)
{
    pdl_enter();
    const long long N = g.N[l];
    GRID_STRIDE(id, N)
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
        double* q0 = fbase_w(g, F_Q0, l) + id;
        if (old == 0 && nw != 0) {
            const Ctx x{l, 0, g.lb};
            double p[M];
            predict<D, M>(g, x, l, c, p);
#pragma unroll
            for (int v = 0; v < M; ++v) q0[v * N] = p[v];
        }
        if (nw == 1) {
            double* qe = fbase_w(g, F_QE, l) + id;
#pragma unroll
            for (int v = 0; v < M; ++v) qe[v * N] = q0[v * N];
        }
        if (g.rc) {
            const long long roff = g.off[l] * g.nf * M;
            for (int r = 0; r < g.nf * M; ++r) {
                g.rc[roff + r * N + id] = 0.0;
                g.rf[roff + r * N + id] = 0.0;
            }
        }
    }
}

// ------------------------------------------------------------ compaction
// Level l owns the blocks [lb.base[l], lb.base[l+1]) of a compaction launch
// over levels lb.lo..lb.hi (NTHREADS cells per block).
struct LevelBlocks {
    int lo, hi;
    int base[LMAX + 2];
};

__device__ __forceinline__ int block_level(const LevelBlocks& b, int blk)
{
    int l = b.lo;
    while (l < b.hi && blk >= b.base[l + 1]) ++l;
    return l;
}

__global__ void k_cmp_count(Grid g, LevelBlocks lbk, int* bc)
{
    pdl_enter();
    const int l = block_level(lbk, blockIdx.x);
    const long long N = g.N[l];
    const long long i = (long long)(blockIdx.x - lbk.base[l]) * blockDim.x + threadIdx.x;
    const int s = i < N ? status(g, l, i) : 0;
    const unsigned bl = __ballot_sync(0xffffffffu, s == 1);
    const unsigned bi = __ballot_sync(0xffffffffu, s == 2);
    __shared__ int wl[NTHREADS / 32], wi[NTHREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        wl[warp] = __popc(bl);
        wi[warp] = __popc(bi);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int a = 0, b = 0;
        for (int w = 0; w < NTHREADS / 32; ++w) {
            a += wl[w];
            b += wi[w];
        }
        bc[2 * blockIdx.x] = a;
        bc[2 * blockIdx.x + 1] = b;
    }
}

// exclusive scan of the per-block counts, one block per level; totals to counts[l]
__global__ void k_cmp_scan(Grid g, LevelBlocks lbk, int* bc)
{
    pdl_enter();
    __shared__ int sa[1024], sb[1024];
    const int l = lbk.lo + blockIdx.x;
    const int b0l = lbk.base[l], nb = lbk.base[l + 1] - b0l;
    const int tid = threadIdx.x;
    const int per = (nb + 1023) / 1024;
    const int b0 = b0l + tid * per, b1 = min(b0 + per, b0l + nb);
    int a = 0, b = 0;
    for (int i = b0; i < b1; ++i) {
        a += bc[2 * i];
        b += bc[2 * i + 1];
    }
    sa[tid] = a;
    sb[tid] = b;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
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
    if (tid == 1023) {
        g.counts[l] = sa[1023];
        g.counts[LMAX + 1 + l] = sb[1023];
    }
}

__global__ void k_cmp_scatter(Grid g, LevelBlocks lbk, const int* bc)
{
    pdl_enter();
    const int l = block_level(lbk, blockIdx.x);
    const long long N = g.N[l];
    const long long i = (long long)(blockIdx.x - lbk.base[l]) * blockDim.x + threadIdx.x;
    const int s = i < N ? status(g, l, i) : 0;
    const unsigned bl = __ballot_sync(0xffffffffu, s == 1);
    const unsigned bi = __ballot_sync(0xffffffffu, s == 2);
    __shared__ int wl[NTHREADS / 32], wi[NTHREADS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        wl[warp] = __popc(bl);
        wi[warp] = __popc(bi);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int a = bc[2 * blockIdx.x], b = bc[2 * blockIdx.x + 1];
        for (int w = 0; w < NTHREADS / 32; ++w) {
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
    if (s == 1) { // the leaf's tile is active
        const long long n = g.n[l];
        const int tx = g.d == 1 ? kTile1X : (g.d == 2 ? kTile2X : kTile3X);
        const int ty = g.d == 2 ? kTile2Y : kTile3Y;
        const long long x = i % n, y = g.d >= 2 ? (i / n) % n : 0, z = g.d == 3 ? i / (n * n) : 0;
        g.tflag[g.toff[l] + x / tx + (long long)g.ntx[l] * (y / ty + (long long)g.nty[l] * (z / kTile3Z))] = 1;
    }
}

// ordered list of the active tiles of level lo + blockIdx.x (one block per level)
__global__ void k_tile_list(Grid g, int lo)
{
    pdl_enter();
    __shared__ int sc[1024];
    const int l = lo + blockIdx.x;
    const int nt = g.ntx[l] * g.nty[l] * g.ntz[l];
    const uint8_t* fl = g.tflag + g.toff[l];
    const int tid = threadIdx.x, per = (nt + 1023) / 1024;
    const int t0 = tid * per, t1 = min(t0 + per, nt);
    int c = 0;
    for (int t = t0; t < t1; ++t) c += fl[t] != 0;
    sc[tid] = c;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const int xo = tid >= o ? sc[tid - o] : 0;
        __syncthreads();
        sc[tid] += xo;
        __syncthreads();
    }
    int pos = sc[tid] - c;
    for (int t = t0; t < t1; ++t)
        if (fl[t]) g.tlist[g.toff[l] + pos++] = t;
    if (tid == 1023) g.counts[2 * (LMAX + 1) + l] = sc[1023];
}

// ------------------------------------------------------------ registers
// conservative correction of the coarse leaves of level l whose step ended:
// q += +-(coarse time-integrated flux - mean of the fine ones) / dx; the
// registers read are cleared for the next step
template <int D>
__global__ void k_reflux(Grid g, int lo, int hi)
{
    pdl_enter();
  for (int l = lo; l <= hi; ++l) {
    const int cnt = g.counts[l];
    const int* list = g.leaves + g.off[l];
    const long long N = g.N[l], Nf = g.N[l + 1];
    const int m = g.m;
    constexpr int NT = 1 << (D - 1);
    GRID_STRIDE(t, cnt)
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
            double* rc = g.rc + g.off[l] * g.nf * m + id;
            double* rf = g.rf + g.off[l + 1] * g.nf * m;
            double* qe = fbase_w(g, F_QE, l) + id;
            const double idx = 1.0 / g.dx[l][k];
            for (int v = 0; v < m; ++v) {
                double sum = 0.0;
                for (int tt = 0; tt < NT; ++tt) {
                    double* r = rf + (long long)(opp * m + v) * Nf + ch[tt];
                    sum += *r;
                    *r = 0.0;
                }
                double* r = rc + (long long)(fi * m + v) * N;
                qe[v * N] += side * (*r - sum * (1.0 / NT)) * idx;
                *r = 0.0;
            }
        }
    }
  }
}

// ------------------------------------------------------------ reductions
__global__ void k_scale(Grid g, int l)
{
    pdl_enter();
    const int cnt = g.counts[l];
    const int* list = g.leaves + g.off[l];
    const long long N = g.N[l];
    double mx[MMAX] = {0.0, 0.0, 0.0, 0.0, 0.0};
    GRID_STRIDE(t, cnt)
    {
        const long long id = list[t];
        if (id < 0 || id >= N) continue;
        for (int v = 0; v < g.m; ++v) mx[v] = fmax(mx[v], fabs(fbase(g, F_Q0, l)[v * N + id]));
    }
    for (int v = 0; v < g.m; ++v) {
        double a = mx[v];
        for (int o = 16; o > 0; o >>= 1) a = fmax(a, __shfl_xor_sync(0xffffffffu, a, o));
        if ((threadIdx.x & 31) == 0 && a > 0.0)
            atomicMax(&g.scale_bits[v], (unsigned long long)__double_as_longlong(a));
    }
}

__global__ void k_finite(Grid g, int l)
{
    pdl_enter();
    const int cnt = g.counts[l];
    const int* list = g.leaves + g.off[l];
    const long long N = g.N[l];
    GRID_STRIDE(t, cnt)
    {
        const long long id = list[t];
        if (id < 0 || id >= N) continue;
        for (int v = 0; v < g.m; ++v)
            if (!isfinite(fbase(g, F_QE, l)[v * N + id])) atomicOr(g.err, ERR_NONFINITE);
    }
}

// fixed-shape partial sums (deterministic): part[block * m + v]
__global__ void k_mass(Grid g, int l, double* part)
{
    pdl_enter();
    __shared__ double sh[NTHREADS];
    const int cnt = g.counts[l];
    const int* list = g.leaves + g.off[l];
    const long long N = g.N[l];
    for (int v = 0; v < g.m; ++v) {
        double acc = 0.0;
        for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < cnt;
             t += (long long)gridDim.x * blockDim.x) {
            const long long id = list[t];
            if (id >= 0 && id < N) acc += fbase(g, F_QE, l)[v * N + id];
        }
        sh[threadIdx.x] = acc;
        __syncthreads();
        for (int o = NTHREADS / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) part[blockIdx.x * g.m + v] = sh[0];
        __syncthreads();
    }
}

__global__ void k_pack(Grid g, int l, long long base, int* keys, double* vals)
{
    pdl_enter();
    const int cnt = g.counts[l];
    const int* list = g.leaves + g.off[l];
    const long long N = g.N[l];
    GRID_STRIDE(t, cnt)
    {
        const long long id = list[t];
        if (id < 0 || id >= N) continue;
        int c[3];
        cell_xyz(g, l, id, c);
        if (keys) {
            int* K = keys + (base + t) * 4;
            K[0] = l;
            K[1] = c[0];
            K[2] = c[1];
            K[3] = c[2];
        }
        if (vals)
            for (int v = 0; v < g.m; ++v) vals[(base + t) * g.m + v] = fbase(g, F_QE, l)[v * N + id];
    }
}

// inverse MR transform onto the finest level, in scratch pyramids T / us:
// bottom-up projection of the leaves' q^{n+1} into internal nodes, then
// top-down prediction of every absent cell from the level above
template <int D>
__global__ void k_uni_up(Grid g, int l, double* T, uint8_t* us)
{
    pdl_enter();
    const long long N = g.N[l];
    const long long Nc = l < g.L ? g.N[l + 1] : 0;
    double* Tl = T + g.off[l] * g.m;
    const double* Tc = l < g.L ? T + g.off[l + 1] * g.m : nullptr;
    GRID_STRIDE(id, N)
    {
        const int s = status(g, l, id);
        us[g.off[l] + id] = s != 0;
        if (s == 1) {
            for (int v = 0; v < g.m; ++v) Tl[v * N + id] = fbase(g, F_QE, l)[v * N + id];
        } else if (s == 2) {
            int c[3];
            cell_xyz(g, l, id, c);
            for (int v = 0; v < g.m; ++v) {
                double acc = 0.0;
                for (int k = 0; k < (1 << D); ++k)
                    acc += Tc[v * Nc + cell_id(g, l + 1, 2 * c[0] + (k & 1), D > 1 ? 2 * c[1] + ((k >> 1) & 1) : 0,
                                                D > 2 ? 2 * c[2] + ((k >> 2) & 1) : 0)];
                Tl[v * N + id] = acc * (1.0 / (1 << D));
            }
        }
    }
}

template <int D>
__global__ void k_uni_down(Grid g, int l, double* T, uint8_t* us)
{
    pdl_enter();
    const long long N = g.N[l], Np = g.N[l - 1];
    double* Tl = T + g.off[l] * g.m;
    const double* Tp = T + g.off[l - 1] * g.m;
    GRID_STRIDE(id, N)
    {
        if (us[g.off[l] + id]) continue;
        int c[3];
        cell_xyz(g, l, id, c);
        const int P[3] = {c[0] >> 1, c[1] >> 1, c[2] >> 1};
        for (int v = 0; v < g.m; ++v) {
            double acc = 0.0;
            FOR3(D, dx, dy, dz)
            {
                int neg = 0;
                const int x = wrap_or_mirror(g, l - 1, 0, P[0] + dx, neg);
                const int y = D > 1 ? wrap_or_mirror(g, l - 1, 1, P[1] + dy, neg) : 0;
                const int z = D > 2 ? wrap_or_mirror(g, l - 1, 2, P[2] + dz, neg) : 0;
                const double w0 = pw(c[0] & 1, dx) * (D > 1 ? pw(c[1] & 1, dy) : 1.0) * (D > 2 ? pw(c[2] & 1, dz) : 1.0);
                const double w = neg ? -w0 : w0;
                acc += w * Tp[v * Np + cell_id(g, l - 1, x, y, z)];
            }
            Tl[v * N + id] = acc;
        }
        us[g.off[l] + id] = 1;
    }
}

// ------------------------------------------------------------ launchers
template <int D>
static void project_d(Launcher& L, int l, int mode)
{
    pdl_launch(k_project<D>, blocks_list(L.g, l), NTHREADS, 0, L.st, L.g, l, mode);
}

void Launcher::project(int l, int mode)
{
    ++n;
    if (g.d == 1) project_d<1>(*this, l, mode);
    else if (g.d == 2) project_d<2>(*this, l, mode);
    else project_d<3>(*this, l, mode);
}

void Launcher::leaf_copy(int lo, int hi, int from, int to)
{
    ++n;
    pdl_launch(k_leaf_copy, blocks_list(g, hi), NTHREADS, 0, st, g, lo, hi, from, to);
}

template <int D, int M>
static void adapt_dm(Launcher& L, int la)
{
    const Grid& g = L.g;
    const int hi = g.L - 1; // levels whose nodes may own children
    pdl_launch(k_detail<D, M>, blocks_list(g, hi), NTHREADS, 0, L.st, g, la, hi);
    pdl_launch(k_desire<D>, blocks_dense(g.N[hi]), NTHREADS, 0, L.st, g, la, hi, la);
    pdl_launch(k_allow<D>, blocks_dense(g.N[hi]), NTHREADS, 0, L.st, g, la, hi, la);
    L.n += 3;
    for (int l = g.L - 1; l > la; --l, ++L.n) pdl_launch(k_close<D>, blocks_dense(g.N[l - 1]), NTHREADS, 0, L.st, g, l);
}

template <int D, int M>
static void apply_dm(Launcher& L, int la)
{
    const Grid& g = L.g;
    for (int l = la; l <= g.L; ++l, ++L.n) pdl_launch(k_apply<D, M>, blocks_dense(g.N[l]), NTHREADS, 0, L.st, g, l, la);
}

#define MRLT_DM_DISPATCH(fn, ...)                                   \
    do {                                                            \
        if (g.d == 1 && g.m == 1) fn<1, 1>(__VA_ARGS__);            \
        else if (g.d == 1) fn<1, 3>(__VA_ARGS__);                   \
        else if (g.d == 2 && g.m == 1) fn<2, 1>(__VA_ARGS__);       \
        else if (g.d == 2) fn<2, 4>(__VA_ARGS__);                   \
        else if (g.m == 1) fn<3, 1>(__VA_ARGS__);                   \
        else fn<3, 5>(__VA_ARGS__);                                 \
    } while (0)

void Launcher::mark_refinements(int la) { MRLT_DM_DISPATCH(adapt_dm, *this, la); }
void Launcher::apply_tree(int la) { MRLT_DM_DISPATCH(apply_dm, *this, la); }

void Launcher::compact(int lo, int hi)
{
    LevelBlocks lbk;
    lbk.lo = lo;
    lbk.hi = hi;
    int total = 0;
    for (int l = lo; l <= hi; ++l) {
        lbk.base[l] = total;
        total += (int)((g.N[l] + NTHREADS - 1) / NTHREADS);
    }
    lbk.base[hi + 1] = total;
    cudaMemsetAsync(g.tflag + g.toff[lo], 0,
                    (size_t)(g.toff[hi] - g.toff[lo]) + (size_t)g.ntx[hi] * g.nty[hi] * g.ntz[hi], st);
    pdl_launch(k_cmp_count, total, NTHREADS, 0, st, g, lbk, bc);
    pdl_launch(k_cmp_scan, hi - lo + 1, 1024, 0, st, g, lbk, bc);
    pdl_launch(k_cmp_scatter, total, NTHREADS, 0, st, g, lbk, (const int*)bc);
    pdl_launch(k_tile_list, hi - lo + 1, 1024, 0, st, g, lo);
    n += 4;
}

void Launcher::reflux(int lo, int hi)
{
    ++n;
    if (g.d == 1) pdl_launch(k_reflux<1>, blocks_list(g, hi), NTHREADS, 0, st, g, lo, hi);
    else if (g.d == 2) pdl_launch(k_reflux<2>, blocks_list(g, hi), NTHREADS, 0, st, g, lo, hi);
    else pdl_launch(k_reflux<3>, blocks_list(g, hi), NTHREADS, 0, st, g, lo, hi);
}

__global__ void k_scale_init(Grid g)
{
    pdl_enter();
    if (threadIdx.x < MMAX) g.scale_bits[threadIdx.x] = (unsigned long long)__double_as_longlong(1e-14);
}

__global__ void k_set_dt(Grid g, double dt)
{
    pdl_enter();
    if (threadIdx.x == 0) *g.dtp = dt;
}

// leaf values from (level, i, j, k) keys: q^n and the end value of each leaf
// (restoring a state saved at a macro-step boundary); a key that is not a
// leaf of the installed tree sets ERR_INDEX
__global__ void k_set_leaves(Grid g, const int* keys, const double* vals, long long n)
{
    pdl_enter();
    GRID_STRIDE(t, n)
    {
        const int* K = keys + 4 * t;
        const int l = K[0];
        if (l < g.lb || l > g.L || K[1] < 0 || K[1] >= g.n[l] || (g.d > 1 && (K[2] < 0 || K[2] >= g.n[l])) ||
            (g.d > 2 && (K[3] < 0 || K[3] >= g.n[l]))) {
            atomicOr(g.err, ERR_INDEX);
            continue;
        }
        const long long id = cell_id(g, l, K[1], g.d > 1 ? K[2] : 0, g.d > 2 ? K[3] : 0);
        if (status(g, l, id) != 1) {
            atomicOr(g.err, ERR_INDEX);
            continue;
        }
        const long long N = g.N[l];
        double* q0 = fbase_w(g, F_Q0, l) + id;
        double* qe = fbase_w(g, F_QE, l) + id;
        for (int v = 0; v < g.m; ++v) q0[v * N] = qe[v * N] = vals[t * g.m + v];
    }
}

void Launcher::set_leaves(const int* keys, const double* vals, long long count)
{
    pdl_launch(k_set_leaves, blocks_dense(count), NTHREADS, 0, st, g, keys, vals, count);
    ++n;
}

void Launcher::scale_init()
{
    pdl_launch(k_scale_init, 1, 32, 0, st, g);
    ++n;
}

void Launcher::set_dt(double dt)
{
    pdl_launch(k_set_dt, 1, 32, 0, st, g, dt);
    ++n;
}

void Launcher::scale(int l)
{
    ++n;
    k_scale<<<blocks_list(g, l), NTHREADS, 0, st>>>(g, l);
}
void Launcher::finite(int l)
{
    ++n;
    k_finite<<<blocks_list(g, l), NTHREADS, 0, st>>>(g, l);
}
void Launcher::mass(int l, double* part)
{
    ++n;
    k_mass<<<MASS_BLOCKS, NTHREADS, 0, st>>>(g, l, part);
}
void Launcher::pack(int l, long long base, int* keys, double* vals)
{
    ++n;
    k_pack<<<blocks_list(g, l), NTHREADS, 0, st>>>(g, l, base, keys, vals);
}
void Launcher::uniform(double* T, uint8_t* us)
{
    for (int l = g.L; l >= g.lb; --l, ++n) {
        if (g.d == 1) k_uni_up<1><<<blocks_dense(g.N[l]), NTHREADS, 0, st>>>(g, l, T, us);
        else if (g.d == 2) k_uni_up<2><<<blocks_dense(g.N[l]), NTHREADS, 0, st>>>(g, l, T, us);
        else k_uni_up<3><<<blocks_dense(g.N[l]), NTHREADS, 0, st>>>(g, l, T, us);
    }
    for (int l = g.lb + 1; l <= g.L; ++l, ++n) {
        if (g.d == 1) k_uni_down<1><<<blocks_dense(g.N[l]), NTHREADS, 0, st>>>(g, l, T, us);
        else if (g.d == 2) k_uni_down<2><<<blocks_dense(g.N[l]), NTHREADS, 0, st>>>(g, l, T, us);
        else k_uni_down<3><<<blocks_dense(g.N[l]), NTHREADS, 0, st>>>(g, l, T, us);
    }
}

} // namespace mrlt

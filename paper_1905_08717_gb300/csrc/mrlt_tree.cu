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

#define GRID_STRIDE(i, n) MRLT_GRID_STRIDE(i, n)

// ------------------------------------------------------------ kernels
// Each kernel waits for its predecessor (programmatic dependent launch) and
// runs one device body of mrlt_tree_dev.cuh over its own grid.
// (T: the storage type of the fields, double or float)
template <class T>
__global__ void k_leaf_copy(const __grid_constant__ Grid g, int lo, int hi, int from, int to)
{
    MRLT_ENTER(g);
    dev_leaf_copy<T>(g, lo, hi, from, to);
}

template <int D, class T>
__global__ void k_project(const __grid_constant__ Grid g, int l, int mode)
{
    MRLT_ENTER(g);
    dev_project<D, T>(g, l, mode);
}

// up-sweep of levels hi..lo in one launch (dev_project_up)
template <int D, class T>
__global__ void k_project_up(const __grid_constant__ Grid g, int hi, int lo, int mode)
{
    MRLT_ENTER(g);
    dev_project_up<D, T>(g, hi, lo, mode);
}

template <int D, int M, class T>
__global__ void k_detail(const __grid_constant__ Grid g, int lo, int hi)
{
    MRLT_ENTER(g);
    dev_detail<D, M, T>(g, lo, hi);
}

// Desired and admissible refinements in one pass: a cell's admissibility
// reads only its own desire bit (set by the same thread, same grid-stride
// order), and desire reads only the detail bits, which admissibility keeps.
// it >= 0: this launch finalises the refinement flags (a remesh at level
// la = L-1 has no closure), so it also checks that the new tree fits.
template <int D>
__global__ void k_mark(const __grid_constant__ Grid g, int lo, int hi, int la, long long it)
{
    MRLT_ENTER(g);
    dev_desire<D>(g, lo, hi, la);
    dev_allow<D>(g, lo, hi, la);
    if (it >= 0) room_decide(g, refined_here(g, la), la, it);
}

// it >= 0: the last closure (level l-1 = la), which also checks that the new
// tree fits; its threads read back the level-la flags they wrote themselves
template <int D>
__global__ void k_close(const __grid_constant__ Grid g, int l, long long it)
{
    MRLT_ENTER(g);
    dev_close<D>(g, l);
    if (it >= 0) room_decide(g, refined_here(g, l - 1), l - 1, it);
}

template <int D, int M, class T>
__global__ void k_apply(const __grid_constant__ Grid g, int l, int la)
{
    MRLT_ENTER(g);
    dev_apply<D, M, T>(g, l, la);
}

// the releases of a remesh and its installation on level la in one launch:
// level la creates no node (its nodes stay; only leaf and internal swap), so
// it takes no slot, and the released nodes (levels above la) are not its
template <int D, int M, class T>
__global__ void k_release_apply(const __grid_constant__ Grid g, int la)
{
    MRLT_ENTER(g);
    dev_release(g, la);
    dev_apply<D, M, T>(g, la, la);
}

// compaction of levels lo..hi: chunks of NTHREADS cells, one block each;
// the tile flags of those levels [t0, t1) cleared for the scatter
__global__ void k_cmp_count(const __grid_constant__ Grid g, LevelChunks lc, int* bc, long long t0, long long t1)
{
    MRLT_ENTER(g);
    chunk_count<NTHREADS>(g, lc, blockIdx.x, bc);
    MRLT_GRID_STRIDE(i, t1 - t0) g.tflag[t0 + i] = 0;
}

// exclusive scan of the per-chunk counts, one block per level
__global__ void k_cmp_scan(const __grid_constant__ Grid g, LevelChunks lc, int* bc)
{
    MRLT_ENTER(g);
    level_scan<1024>(g, lc, lc.lo + blockIdx.x, bc);
}

__global__ void k_cmp_scatter(const __grid_constant__ Grid g, LevelChunks lc, const int* bc)
{
    MRLT_ENTER(g);
    chunk_scatter<NTHREADS>(g, lc, blockIdx.x, bc);
}

// ordered list of the active tiles of level lo + blockIdx.x (one block per level)
__global__ void k_tile_list(const __grid_constant__ Grid g, int lo)
{
    MRLT_ENTER(g);
    level_tile_list<1024>(g, lo + blockIdx.x);
}

template <int D, class T>
__global__ void k_reflux(const __grid_constant__ Grid g, int lo, int hi)
{
    MRLT_ENTER(g);
    dev_reflux<D, T>(g, lo, hi);
}

// ------------------------------------------------------------ reductions
template <class T>
__global__ void k_scale(const __grid_constant__ Grid g, int l)
{
    MRLT_ENTER(g);
    dev_scale<T>(g, l, l);
}

template <class T>
__global__ void k_finite(const __grid_constant__ Grid g, int l)
{
    MRLT_ENTER(g);
    dev_finite<T>(g, l, l);
}

// fixed-shape partial sums (deterministic): part[block * m + v]
template <class T>
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
            if (id >= 0 && id < N) acc += double(nd<T>(g, F_QE, slot_of(g, l, id))[v]);
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

template <class T>
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
            for (int v = 0; v < g.m; ++v) vals[(base + t) * g.m + v] = double(nd<T>(g, F_QE, slot_of(g, l, id))[v]);
    }
}

// inverse MR transform onto the finest level, in scratch pyramids T / us:
// bottom-up projection of the leaves' q^{n+1} into internal nodes, then
// top-down prediction of every absent cell from the level above
template <int D, class F>
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
            for (int v = 0; v < g.m; ++v) Tl[v * N + id] = double(nd<F>(g, F_QE, slot_of(g, l, id))[v]);
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
            MRLT_FOR3(D, dx, dy, dz)
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
template <int D, class T>
static void project_d(Launcher& L, int l, int mode)
{
    pdl_launch(k_project<D, T>, blocks_list(L.g, l), NTHREADS, 0, L.st, L.g, l, mode);
}

// a kernel template of the fields' storage type: float in the mixed mode
#define MRLT_T_DISPATCH(fn, ...)              \
    do {                                      \
        if (g.prec) fn<float>(__VA_ARGS__);   \
        else fn<double>(__VA_ARGS__);         \
    } while (0)

void Launcher::project(int l, int mode)
{
    ++n;
    if (g.d == 1) g.prec ? project_d<1, float>(*this, l, mode) : project_d<1, double>(*this, l, mode);
    else if (g.d == 2) g.prec ? project_d<2, float>(*this, l, mode) : project_d<2, double>(*this, l, mode);
    else g.prec ? project_d<3, float>(*this, l, mode) : project_d<3, double>(*this, l, mode);
}

// Up-sweep hi -> lo in groups of at most 6 / d + 1 levels per launch: a group
// [glo, ghi] has 2^{d (ghi - glo)} <= 64 descendants per top node, so two top
// nodes fit the NTHREADS = 128 threads of a CTA.
template <int D, class T>
static void project_up_d(Launcher& L, int hi, int lo, int mode)
{
    constexpr int kDepth = 6 / D;
    static_assert((1 << (D * kDepth)) * 2 <= NTHREADS, "two top nodes per CTA");
    for (int ghi = hi; ghi >= lo;) {
        const int glo = ghi - kDepth > lo ? ghi - kDepth : lo;
        if (glo == ghi) {
            project_d<D, T>(L, ghi, mode);
        } else {
            const int tops = NTHREADS >> (D * (ghi - glo));
            long long b = (L.g.N[glo] + tops - 1) / tops;
            if (b > 1216) b = 1216;
            pdl_launch(k_project_up<D, T>, (int)b, NTHREADS, 0, L.st, L.g, ghi, glo, mode);
        }
        ++L.n;
        ghi = glo - 1;
    }
}

void Launcher::project_up(int hi, int lo, int mode)
{
    if (hi < lo) return;
    if (g.d == 1) g.prec ? project_up_d<1, float>(*this, hi, lo, mode) : project_up_d<1, double>(*this, hi, lo, mode);
    else if (g.d == 2) g.prec ? project_up_d<2, float>(*this, hi, lo, mode) : project_up_d<2, double>(*this, hi, lo, mode);
    else g.prec ? project_up_d<3, float>(*this, hi, lo, mode) : project_up_d<3, double>(*this, hi, lo, mode);
}

template <class T>
static void leaf_copy_t(Launcher& L, int lo, int hi, int from, int to)
{
    pdl_launch(k_leaf_copy<T>, blocks_list(L.g, hi), NTHREADS, 0, L.st, L.g, lo, hi, from, to);
}

void Launcher::leaf_copy(int lo, int hi, int from, int to)
{
    ++n;
    MRLT_T_DISPATCH(leaf_copy_t, *this, lo, hi, from, to);
}

template <int D, int M>
static void adapt_dm(Launcher& L, int la, long long it)
{
    const Grid& g = L.g;
    const int hi = g.L - 1; // levels whose nodes may own children
    if (g.prec) pdl_launch(k_detail<D, M, float>, blocks_list(g, hi), NTHREADS, 0, L.st, g, la, hi);
    else pdl_launch(k_detail<D, M, double>, blocks_list(g, hi), NTHREADS, 0, L.st, g, la, hi);
    pdl_launch(k_mark<D>, blocks_dense(g.N[hi]), NTHREADS, 0, L.st, g, la, hi, la, la == hi ? it : -1LL);
    L.n += 2;
    for (int l = g.L - 1; l > la; --l, ++L.n)
        pdl_launch(k_close<D>, blocks_dense(g.N[l - 1]), NTHREADS, 0, L.st, g, l, l == la + 1 ? it : -1LL);
}


template <int D, int M>
static void apply_dm(Launcher& L, int la)
{
    const Grid& g = L.g;
    const int b0 = blocks_list(g, g.L), b1 = blocks_dense(g.N[la]);
    if (g.prec) pdl_launch(k_release_apply<D, M, float>, b0 > b1 ? b0 : b1, NTHREADS, 0, L.st, g, la);
    else pdl_launch(k_release_apply<D, M, double>, b0 > b1 ? b0 : b1, NTHREADS, 0, L.st, g, la);
    ++L.n;
    for (int l = la + 1; l <= g.L; ++l, ++L.n) {
        if (g.prec) pdl_launch(k_apply<D, M, float>, blocks_dense(g.N[l]), NTHREADS, 0, L.st, g, l, la);
        else pdl_launch(k_apply<D, M, double>, blocks_dense(g.N[l]), NTHREADS, 0, L.st, g, l, la);
    }
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

void Launcher::mark_refinements(int la, long long it) { MRLT_DM_DISPATCH(adapt_dm, *this, la, it); }
void Launcher::apply_tree(int la) { MRLT_DM_DISPATCH(apply_dm, *this, la); }

void Launcher::compact(int lo, int hi)
{
    LevelChunks lbk;
    lbk.lo = lo;
    lbk.hi = hi;
    int total = 0;
    for (int l = lo; l <= hi; ++l) {
        lbk.base[l] = total;
        total += (int)((g.N[l] + NTHREADS - 1) / NTHREADS);
    }
    lbk.base[hi + 1] = total;
    const long long t0 = g.toff[lo], t1 = g.toff[hi] + (long long)g.ntx[hi] * g.nty[hi] * g.ntz[hi];
    pdl_launch(k_cmp_count, total, NTHREADS, 0, st, g, lbk, bc, t0, t1);
    pdl_launch(k_cmp_scan, hi - lo + 1, 1024, 0, st, g, lbk, bc);
    pdl_launch(k_cmp_scatter, total, NTHREADS, 0, st, g, lbk, (const int*)bc);
    pdl_launch(k_tile_list, hi - lo + 1, 1024, 0, st, g, lo);
    n += 4;
}

template <class T>
static void reflux_t(Launcher& L, int lo, int hi)
{
    const Grid& g = L.g;
    if (g.d == 1) pdl_launch(k_reflux<1, T>, blocks_list(g, hi), NTHREADS, 0, L.st, g, lo, hi);
    else if (g.d == 2) pdl_launch(k_reflux<2, T>, blocks_list(g, hi), NTHREADS, 0, L.st, g, lo, hi);
    else pdl_launch(k_reflux<3, T>, blocks_list(g, hi), NTHREADS, 0, L.st, g, lo, hi);
}

void Launcher::reflux(int lo, int hi)
{
    ++n;
    MRLT_T_DISPATCH(reflux_t, *this, lo, hi);
}

__global__ void k_scale_init(Grid g)
{
    MRLT_ENTER(g);
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
template <class T>
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
        const int sl = slot_of(g, l, id);
        T* q0 = nd<T>(g, F_Q0, sl);
        T* qe = nd<T>(g, F_QE, sl);
        for (int v = 0; v < g.m; ++v) q0[v] = qe[v] = T(vals[t * g.m + v]);
    }
}

void Launcher::set_leaves(const int* keys, const double* vals, long long count)
{
    if (g.prec) pdl_launch(k_set_leaves<float>, blocks_dense(count), NTHREADS, 0, st, g, keys, vals, count);
    else pdl_launch(k_set_leaves<double>, blocks_dense(count), NTHREADS, 0, st, g, keys, vals, count);
    ++n;
}

// finest-level data (host layout [v][cell], uploaded as double) stored in
// q^n of the finest nodes, in the fields' type
template <class T>
__global__ void k_store_finest(Grid g, const double* src)
{
    pdl_enter();
    const long long N = g.N[g.L];
    GRID_STRIDE(id, N)
    {
        T* q0 = nd<T>(g, F_Q0, slot_of(g, g.L, id));
        for (int v = 0; v < g.m; ++v) q0[v] = T(src[v * N + id]);
    }
}

void Launcher::store_finest(const double* src)
{
    if (g.prec) pdl_launch(k_store_finest<float>, blocks_dense(g.N[g.L]), NTHREADS, 0, st, g, src);
    else pdl_launch(k_store_finest<double>, blocks_dense(g.N[g.L]), NTHREADS, 0, st, g, src);
    ++n;
}

// every cell of levels lb..L a node in slot 1 + (its offset in the
// pyramid): the full tree of a new solver; the free stack holds the rest
__global__ void k_slots_full(Grid g, long long ntot)
{
    pdl_enter();
    GRID_STRIDE(i, ntot) g.slot[g.off[g.lb] + i] = (int)(1 + i);
    const long long nfree = g.cap - 1 - ntot;
    GRID_STRIDE(k, nfree) g.fstack[k] = (int)(g.cap - 1 - k);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        g.ftop[0] = (int)nfree;
        g.ftop[1] = 0;
    }
}

void Launcher::slots_full(long long ntot)
{
    pdl_launch(k_slots_full, blocks_dense(ntot), NTHREADS, 0, st, g, ntot);
    ++n;
}

// Refinement flags over cells [from, to), added into *out: after the
// closure of an adaptation at level la every flagged cell of levels
// la..L-1 owns 2^d nodes of the new tree.
__global__ void k_count_ref(const __grid_constant__ Grid g, long long from, long long to, int* out)
{
    MRLT_ENTER(g);
    int c = 0;
    GRID_STRIDE(i, to - from) c += (g.flag[from + i] & FL_REF) ? 1 : 0;
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

void Launcher::count_refined(int la, int* out)
{
    cudaMemsetAsync(out, 0, sizeof(int), st);
    const long long from = g.off[la], to = g.off[g.L];
    pdl_launch(k_count_ref, blocks_dense(to - from), NTHREADS, 0, st, g, from, to, out);
    ++n;
}


// Compacting copy into node arrays of a new capacity: the nodes of level l
// (leaves, then internal nodes, in list order) take the consecutive slots
// from base[l] + 1; their fields and registers are copied from the old
// arrays (`from`), the slot map rewritten.  The free stack of the new arrays
// holds every slot above the nodes.
template <class T>
__global__ void k_renumber(Grid g, Grid from, LevelChunks base, long long used)
{
    pdl_enter();
    for (int l = g.lb; l <= g.L; ++l) {
        const long long N = g.N[l];
        const int nl = g.counts[l], ni = g.counts[LMAX + 1 + l];
        GRID_STRIDE(t, nl + ni)
        {
            const long long id = t < nl ? g.leaves[g.off[l] + t] : g.inner[g.off[l] + t - nl];
            if (id < 0 || id >= N) {
                atomicOr(g.err, ERR_INDEX);
                continue;
            }
            const int os = slot_of(from, l, id), ns = (int)(1 + base.base[l] + t);
            for (int f = 0; f < NFIELD; ++f) {
                const T* a = nd<T>(from, f, os);
                T* b = nd<T>(g, f, ns);
                for (int v = 0; v < g.m; ++v) b[v] = a[v];
            }
            if (g.rg) {
                const double* a = regs(from.rg, from, os);
                double* b = regs(g.rg, g, ns);
                for (int r = 0; r < g.nf * g.m; ++r) b[r] = a[r];
            }
            g.slot[g.off[l] + id] = ns;
        }
    }
    const long long nfree = g.cap - 1 - used;
    GRID_STRIDE(k, nfree) g.fstack[k] = (int)(g.cap - 1 - k);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        g.ftop[0] = (int)nfree;
        g.ftop[1] = 0;
    }
}

void Launcher::renumber(const Grid& from, const int* counts_host, long long used)
{
    LevelChunks base;
    base.lo = g.lb;
    base.hi = g.L;
    int acc = 0;
    for (int l = g.lb; l <= g.L; ++l) {
        base.base[l] = acc;
        acc += counts_host[l] + counts_host[LMAX + 1 + l];
    }
    base.base[g.L + 1] = acc;
    long long cnt = used > g.cap - 1 - used ? used : g.cap - 1 - used;
    if (g.prec) pdl_launch(k_renumber<float>, blocks_dense(cnt), NTHREADS, 0, st, g, from, base, used);
    else pdl_launch(k_renumber<double>, blocks_dense(cnt), NTHREADS, 0, st, g, from, base, used);
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
    if (g.prec) k_scale<float><<<blocks_list(g, l), NTHREADS, 0, st>>>(g, l);
    else k_scale<double><<<blocks_list(g, l), NTHREADS, 0, st>>>(g, l);
}
void Launcher::finite(int l)
{
    ++n;
    if (g.prec) k_finite<float><<<blocks_list(g, l), NTHREADS, 0, st>>>(g, l);
    else k_finite<double><<<blocks_list(g, l), NTHREADS, 0, st>>>(g, l);
}
void Launcher::mass(int l, double* part)
{
    ++n;
    if (g.prec) k_mass<float><<<MASS_BLOCKS, NTHREADS, 0, st>>>(g, l, part);
    else k_mass<double><<<MASS_BLOCKS, NTHREADS, 0, st>>>(g, l, part);
}
void Launcher::pack(int l, long long base, int* keys, double* vals)
{
    ++n;
    if (g.prec) k_pack<float><<<blocks_list(g, l), NTHREADS, 0, st>>>(g, l, base, keys, vals);
    else k_pack<double><<<blocks_list(g, l), NTHREADS, 0, st>>>(g, l, base, keys, vals);
}
void Launcher::uniform(double* T, uint8_t* us)
{
    for (int l = g.L; l >= g.lb; --l, ++n) {
        const int nb = blocks_dense(g.N[l]);
        if (g.prec) {
            if (g.d == 1) k_uni_up<1, float><<<nb, NTHREADS, 0, st>>>(g, l, T, us);
            else if (g.d == 2) k_uni_up<2, float><<<nb, NTHREADS, 0, st>>>(g, l, T, us);
            else k_uni_up<3, float><<<nb, NTHREADS, 0, st>>>(g, l, T, us);
        } else {
            if (g.d == 1) k_uni_up<1, double><<<nb, NTHREADS, 0, st>>>(g, l, T, us);
            else if (g.d == 2) k_uni_up<2, double><<<nb, NTHREADS, 0, st>>>(g, l, T, us);
            else k_uni_up<3, double><<<nb, NTHREADS, 0, st>>>(g, l, T, us);
        }
    }
    for (int l = g.lb + 1; l <= g.L; ++l, ++n) {
        if (g.d == 1) k_uni_down<1><<<blocks_dense(g.N[l]), NTHREADS, 0, st>>>(g, l, T, us);
        else if (g.d == 2) k_uni_down<2><<<blocks_dense(g.N[l]), NTHREADS, 0, st>>>(g, l, T, us);
        else k_uni_down<3><<<blocks_dense(g.N[l]), NTHREADS, 0, st>>>(g, l, T, us);
    }
}

} // namespace mrlt

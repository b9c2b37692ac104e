// mrlt_macro.cuh -- the persistent macro-step kernel: a run of fine
// iterations of one solver (Alg. 3 in LT mode, the global-step iteration of
// MR/RK otherwise) in ONE cooperative launch.  Every CTA of the grid is
// resident; the phases of an iteration that the kernel-per-phase path
// launches one after another (leaf copy, projections and refreshes per level,
// the adaptation passes, compaction, stage sweeps per level, reflux) are
// separated by a grid-wide barrier instead of a kernel boundary.  Each phase
// runs the same device body (mrlt_tree_dev.cuh, stage_tiles) over the same
// data in the same order, so the results are bitwise those of the
// kernel-per-phase path; only the launch and dependency latency between
// phases is gone.
//
// The barrier waits are bounded: a CTA that has waited longer than the
// launch's limit (or sees that another CTA gave up) sets ERR_TIMEOUT and the
// whole grid returns; the host reports MR_E_TIMEOUT and the context stays
// usable.  Cooperative launch guarantees that all CTAs are co-resident, so a
// correct run never reaches the limit.
#pragma once
#include <atomic>

#include "mrlt_stage.cuh"
#include "mrlt_tree_dev.cuh"

namespace mrlt {


// Arguments of one macro-step kernel launch.  (The fields are stored in the
// stage arithmetic type R: double, or float in the mixed-precision mode.)
struct MacroArgs {
    long long n0, n1;             // fine iterations [n0, n1) of the macro step
    long long nit;                // fine iterations per macro step, 2^{L - min level}
    int adapt_mode;               // MR_ADAPT_*: never / at n = 0 / every iteration
    int reg;                      // flux registers in use (LT mode with reflux)
    int end_of_macro;             // n1 == nit: finiteness check and CFL wave reduction at the end
    unsigned* bar;                // grid barrier [arrivals, generation], zero at launch
    unsigned long long limit_ns;  // longest barrier wait before giving up
    unsigned long long* stamps;   // profiling: (tag, globaltimer ns) at the start of each phase, or null
    int* nstamps;                 // number of stamps written
    int stamp_cap;
    int* bc;                      // compaction scratch, 2 ints per chunk of a level range
};

// phase tags of the profiling stamps: kind << 8 | level
enum PhaseKind { PH_TREE = 0, PH_STAGE1 = 1, PH_STAGE2 = 2, PH_STAGE3 = 3, PH_ADAPT = 4, PH_END = 15 };

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid-wide barrier over the gridDim.x CTAs of the launch (sense by
// generation count).  Thread 0 of each CTA publishes the CTA's writes
// (__threadfence after the CTA barrier), arrives, and the last arriver resets
// the count and releases the next generation; the others poll the
// generation with acquire loads.  Returns false, for every thread of the CTA,
// when the wait gave up.
// `arrivals` is the number of CTAs the barrier waits for: gridDim.x.
__device__ __forceinline__ bool grid_sync(unsigned* bar, unsigned& gen, int* err, unsigned long long limit_ns,
                                          unsigned arrivals)
{
    __syncthreads();
    int ok = 1;
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned g0 = gen;
        if (atomicAdd(&bar[0], 1u) == arrivals - 1) {
            atomicExch(&bar[0], 0u);
            __threadfence();
            atomicExch(&bar[1], g0 + 1u);
        } else {
            const unsigned long long t0 = global_ns();
            while (ld_acquire_gpu(&bar[1]) == g0) {
                if (*(volatile int*)err & ERR_TIMEOUT) {
                    ok = 0;
                    break;
                }
                if (global_ns() - t0 > limit_ns) {
                    atomicOr(err, ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        gen = g0 + 1u;
    }
    return __syncthreads_and(threadIdx.x == 0 ? ok : 1) != 0;
}

__device__ __forceinline__ int level_min_dev(const Grid& g, long long n)
{
    for (int l = g.lb; l <= g.L; ++l)
        if ((n & ((1LL << (g.L - l)) - 1)) == 0) return l;
    return g.L;
}

__device__ __forceinline__ double rk_weight(const Grid& g, int s)
{
    if (g.rk == 2) return 0.5;
    return s == 3 ? 2.0 / 3.0 : 1.0 / 6.0;
}

// Out-of-line phases of the macro-step kernel: each body is compiled once per
// instantiation however many call sites the iteration has (compile time and
// code size), at the cost of one call per phase.
template <int EQ, int D, class R>
__device__ __noinline__ void mph_stage(const Grid& g, int lo, int hi, int s, int lmin, double b, int reg,
                                       unsigned char* smem)
{
    stage_tiles<EQ, D, R>(g, lo, hi, s, lmin, b, reg, smem);
}
template <int D, class T>
__device__ __noinline__ void mph_project(const Grid& g, int l, int mode)
{
    dev_project<D, T>(g, l, mode);
}
template <int D, int M, class T>
__device__ __noinline__ void mph_detail(const Grid& g, int lo, int hi)
{
    dev_detail<D, M, T>(g, lo, hi);
}
template <int D>
__device__ __noinline__ void mph_desire(const Grid& g, int lo, int hi, int la)
{
    dev_desire<D>(g, lo, hi, la);
}
template <int D>
__device__ __noinline__ void mph_allow(const Grid& g, int lo, int hi, int la)
{
    dev_allow<D>(g, lo, hi, la);
}
template <int D>
__device__ __noinline__ void mph_close(const Grid& g, int l)
{
    dev_close<D>(g, l);
}
template <int D, int M, class T>
__device__ __noinline__ void mph_apply(const Grid& g, int l, int la)
{
    dev_apply<D, M, T>(g, l, la);
}
template <int D, class T>
__device__ __noinline__ void mph_reflux(const Grid& g, int lo, int hi)
{
    dev_reflux<D, T>(g, lo, hi);
}
template <int EQ, int D, class T>
__device__ __noinline__ void mph_end(const Grid& g, int lo, int hi)
{
    dev_finite<T>(g, lo, hi);
    dev_wave<EQ, D, T>(g, lo, hi);
}

template <int EQ, int D, class R>
__global__ void __launch_bounds__(Tile<D>::THREADS)
k_macro(const __grid_constant__ Grid g, MacroArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int M = EQ == 2 ? D + 2 : 1;
    constexpr int NT = Tile<D>::THREADS;
    const int L = g.L, lb = g.lb;
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
    unsigned gen = 0;
    int nst = 0;
    // profiling: the start of every phase, tagged kind << 8 | level
    auto phase = [&](int kind, int level) {
        if (a.stamps && lead && nst < a.stamp_cap) {
            a.stamps[2 * nst] = (unsigned long long)(kind << 8 | level);
            a.stamps[2 * nst + 1] = global_ns();
            ++nst;
            *a.nstamps = nst;
        }
    };
#define MRLT_SYNC()                                                 \
    do {                                                            \
        if (!grid_sync(a.bar, gen, g.err, a.limit_ns, gridDim.x)) return; \
    } while (0)

    if (lead && a.end_of_macro) *g.wmax = 0ull; // the CFL reduction of the last phase starts from 0
    for (long long n = a.n0; n < a.n1; ++n) {
        const int lmin = g.gts ? lb : level_min_dev(g, n);
        const bool adapt_now =
            (a.adapt_mode == 2 || (a.adapt_mode == 1 && n == 0)) && lmin < L; // Algs. 1-2 on levels >= lmin
        // begin the step of the active levels: q^n := end value of the leaves,
        // internal nodes by projection (Eq. 3)
        phase(PH_TREE, L);
        if (adapt_now && lmin == lb && lead)
            for (int v = 0; v < MMAX; ++v) g.scale_bits[v] = (unsigned long long)__double_as_longlong(1e-14);
        dev_leaf_copy<R>(g, lmin, L, F_QE, F_Q0);
        MRLT_SYNC();
        for (int l = L - 1; l >= lmin; --l) {
            phase(PH_TREE, l);
            mph_project<D, R>(g, l, PM_Q0);
            MRLT_SYNC();
        }
        if (adapt_now) { // restricted remesh of levels >= la = lmin (Sec. 4)
            const int la = lmin;
            phase(PH_ADAPT, 0);
            if (la == lb) dev_scale<R>(g, lb, L);
            dev_clear_flags(g, g.off[la], g.off[L] + g.N[L]);
            MRLT_SYNC();
            phase(PH_ADAPT, 1);
            mph_detail<D, M, R>(g, la, L - 1);
            MRLT_SYNC();
            phase(PH_ADAPT, 2);
            mph_desire<D>(g, la, L - 1, la);
            MRLT_SYNC();
            phase(PH_ADAPT, 3);
            mph_allow<D>(g, la, L - 1, la);
            MRLT_SYNC();
            for (int l = L - 1; l > la; --l) {
                phase(PH_ADAPT, 4);
                mph_close<D>(g, l);
                MRLT_SYNC();
            }
            phase(PH_ADAPT, 5);
            dev_release(g, la); // slots of removed nodes back on the free stack
            MRLT_SYNC();
            for (int l = la; l <= L; ++l) {
                phase(PH_ADAPT, 5);
                mph_apply<D, M, R>(g, l, la);
                MRLT_SYNC();
            }
            // leaf, node and active-tile lists of levels la..L (chunks of NT cells)
            LevelChunks lc;
            lc.lo = la;
            lc.hi = L;
            int total = 0;
            for (int l = la; l <= L; ++l) {
                lc.base[l] = total;
                total += (int)((g.N[l] + NT - 1) / NT);
            }
            lc.base[L + 1] = total;
            phase(PH_ADAPT, 6);
            {
                const long long t0 = g.toff[la], t1 = g.toff[L] + (long long)g.ntx[L] * g.nty[L] * g.ntz[L];
                MRLT_GRID_STRIDE(i, t1 - t0) g.tflag[t0 + i] = 0;
            }
            for (int c = blockIdx.x; c < total; c += gridDim.x) chunk_count<NT>(g, lc, c, a.bc);
            MRLT_SYNC();
            phase(PH_ADAPT, 7);
            for (int l = la + blockIdx.x; l <= L; l += gridDim.x) level_scan<NT>(g, lc, l, a.bc);
            MRLT_SYNC();
            phase(PH_ADAPT, 8);
            for (int c = blockIdx.x; c < total; c += gridDim.x) chunk_scatter<NT>(g, lc, c, a.bc);
            MRLT_SYNC();
            phase(PH_ADAPT, 9);
            for (int l = la + blockIdx.x; l <= L; l += gridDim.x) level_tile_list<NT>(g, l);
            MRLT_SYNC();
            for (int l = L - 1; l >= la; --l) {
                phase(PH_ADAPT, 10);
                mph_project<D, R>(g, l, PM_Q0);
                MRLT_SYNC();
            }
        }
        if (g.gts) { // MR/RK: every level at the same instant, one phase per stage
            for (int s = 1; s <= g.rk; ++s) {
                if (s > 1)
                    for (int l = L - 1; l >= lb; --l) {
                        phase(PH_TREE, l);
                        mph_project<D, R>(g, l, s == 2 ? PM_Q1 : PM_Q2);
                        MRLT_SYNC();
                    }
                phase(PH_STAGE1 + s - 1, L);
                mph_stage<EQ, D, R>(g, lb, L, s, lb, rk_weight(g, s), 0, smem);
                MRLT_SYNC();
            }
            continue;
        }
        if (lmin > lb) { // Alg. 3 / Sec. 4.3: the mid-step level lmin - 1
            phase(PH_TREE, lmin - 1);
            mph_project<D, R>(g, lmin - 1, PM_MID);
            MRLT_SYNC();
        }
        // first RK stage on every active level (independent levels: one phase)
        phase(PH_STAGE1, L);
        mph_stage<EQ, D, R>(g, lmin, L, 1, lmin, rk_weight(g, 1), a.reg, smem);
        MRLT_SYNC();
        for (int l = L - 1; l >= lmin; --l) { // Alg. 8
            phase(PH_TREE, l);
            mph_project<D, R>(g, l, PM_REF2);
            MRLT_SYNC();
        }
        for (int l = L; l >= lmin; --l) { // Alg. 5 with the Alg. 4 projections
            if (l < L) {
                phase(PH_TREE, l);
                mph_project<D, R>(g, l, PM_PRJ2);
                MRLT_SYNC();
            }
            phase(PH_STAGE2, l);
            mph_stage<EQ, D, R>(g, l, l, 2, lmin, rk_weight(g, 2), a.reg, smem);
            MRLT_SYNC();
        }
        if (g.rk == 3) {
            for (int l = L - 1; l >= lmin; --l) { // Alg. 9
                phase(PH_TREE, l);
                mph_project<D, R>(g, l, PM_REF3);
                MRLT_SYNC();
            }
            for (int l = L; l >= lmin; --l) { // Alg. 7 with the Alg. 6 projections
                if (l < L) {
                    phase(PH_TREE, l);
                    mph_project<D, R>(g, l, PM_PRJ3);
                    MRLT_SYNC();
                }
                phase(PH_STAGE3, l);
                mph_stage<EQ, D, R>(g, l, l, 3, lmin, rk_weight(g, 3), a.reg, smem);
                MRLT_SYNC();
            }
        }
        if (a.reg) { // levels whose step ends with this iteration: apply and clear registers
            const int lc = (n + 1 == a.nit) ? lb : level_min_dev(g, n + 1);
            if (lc < L) {
                phase(PH_TREE, lc);
                mph_reflux<D, R>(g, lc, L - 1);
                MRLT_SYNC();
            }
        }
    }
    if (a.end_of_macro) { // after the macro step: finiteness check and CFL wave speed
        phase(PH_TREE, lb);
        mph_end<EQ, D, R>(g, lb, L);
    }
    phase(PH_END, 0);
#undef MRLT_SYNC
}

// One cooperative launch of k_macro over the device's resident capacity for
// the instantiation (occupancy API, once per device), capped by g.gcap when
// that is set.  Returns 1, or -1 when the kernel cannot be set up or
// launched; a == nullptr only sets it up.
template <int EQ, int D, class R>
static int macro_dispatch(const Grid& g, cudaStream_t st, const MacroArgs* a)
{
    using S = TileShape<EQ, D, R>;
    constexpr int kMaxDev = 64;
    static std::atomic<int> resident[kMaxDev] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return -1;
    if (!resident[dev].load()) {
        int coop = 0, per_sm = 0, sms = 0;
        if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop ||
            cudaFuncSetAttribute(k_macro<EQ, D, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM) !=
                cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_macro<EQ, D, R>, S::NT, S::SMEM) !=
                cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || per_sm < 1)
            return -1;
        resident[dev].store(per_sm * sms);
    }
    if (!a) return 0;
    int grid = resident[dev].load();
    if (g.gcap > 0 && grid > g.gcap) grid = g.gcap;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(S::NT);
    cfg.dynamicSmemBytes = S::SMEM;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_macro<EQ, D, R>, g, *a) == cudaSuccess ? 1 : -1;
}

// macro-step launcher of one equation (all dimensions, both precisions),
// defined beside the stage launchers in mrlt_stage_eq.cu
template <int EQ>
int launch_macro_eq(const Grid& g, cudaStream_t st, const MacroArgs* a);
template <> int launch_macro_eq<0>(const Grid&, cudaStream_t, const MacroArgs*);
template <> int launch_macro_eq<1>(const Grid&, cudaStream_t, const MacroArgs*);
template <> int launch_macro_eq<2>(const Grid&, cudaStream_t, const MacroArgs*);
template <> int launch_macro_eq<3>(const Grid&, cudaStream_t, const MacroArgs*);

} // namespace mrlt

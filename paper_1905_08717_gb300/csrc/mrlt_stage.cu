// mrlt_stage.cu -- stage launch dispatch by equation, and the CFL wave-speed
// reduction.  The stage kernels themselves are in mrlt_stage.cuh, instantiated
// per equation by mrlt_stage_eq.cu.
#include "mrlt_macro.cuh"

namespace mrlt {

// largest sum of characteristic speeds over the leaves of level l (CFL step)
template <int EQ, int D, class T>
__global__ void __launch_bounds__(NTHREADS) k_wave(const __grid_constant__ Grid g, int l)
{
    pdl_enter();
    dev_wave<EQ, D, T>(g, l, l);
}

int launch_stage(const Grid& g, cudaStream_t st, int lo, int hi, int s, int lmin, double b, int reg)
{
    switch (g.eq) {
    case 0: return launch_stage_eq<0>(g, st, lo, hi, s, lmin, b, reg);
    case 1: return launch_stage_eq<1>(g, st, lo, hi, s, lmin, b, reg);
    case 2: return launch_stage_eq<2>(g, st, lo, hi, s, lmin, b, reg);
    case 3: return launch_stage_eq<3>(g, st, lo, hi, s, lmin, b, reg);
    default: return 0;
    }
}

int launch_macro(const Grid& g, cudaStream_t st, const MacroArgs* a)
{
    switch (g.eq) {
    case 0: return launch_macro_eq<0>(g, st, a);
    case 1: return launch_macro_eq<1>(g, st, a);
    case 2: return launch_macro_eq<2>(g, st, a);
    case 3: return launch_macro_eq<3>(g, st, a);
    default: return -1;
    }
}

// Self-test of the bounded grid barrier: `ctas` CTAs wait at one barrier
// that expects ctas + missing arrivals.  With missing > 0 nobody releases it:
// every CTA gives up after limit_ns and ERR_TIMEOUT is set in *err.
__global__ void k_grid_wait_test(unsigned* bar, int* err, unsigned long long limit_ns, unsigned missing)
{
    unsigned gen = 0;
    grid_sync(bar, gen, err, limit_ns, gridDim.x + missing);
}

int launch_grid_wait_test(cudaStream_t st, int ctas, int missing, unsigned long long limit_ns, unsigned* bar,
                          int* err)
{
    k_grid_wait_test<<<ctas, 32, 0, st>>>(bar, err, limit_ns, (unsigned)missing);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

void launch_wave(const Grid& g, cudaStream_t st, int l)
{
#define MRLT_CASE(E, DD)                                                                         \
    if (g.eq == E && g.d == DD) {                                                                \
        if (g.prec) k_wave<E, DD, float><<<grid_for(g, l), NTHREADS, 0, st>>>(g, l);            \
        else k_wave<E, DD, double><<<grid_for(g, l), NTHREADS, 0, st>>>(g, l);                  \
        return;                                                                                  \
    }
    MRLT_CASE(0, 1) MRLT_CASE(0, 2) MRLT_CASE(0, 3)
    MRLT_CASE(1, 1) MRLT_CASE(1, 2) MRLT_CASE(1, 3)
    MRLT_CASE(2, 1) MRLT_CASE(2, 2) MRLT_CASE(2, 3)
    MRLT_CASE(3, 1) MRLT_CASE(3, 2) MRLT_CASE(3, 3)
#undef MRLT_CASE
}

} // namespace mrlt

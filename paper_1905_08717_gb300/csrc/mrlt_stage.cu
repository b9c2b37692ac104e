// mrlt_stage.cu -- stage launch dispatch by equation, and the CFL wave-speed
// reduction.  The stage kernels themselves are in mrlt_stage.cuh, instantiated
// per equation by mrlt_stage_eq.cu.
#include "mrlt_stage.cuh"

namespace mrlt {

// largest sum of characteristic speeds over the leaves of level l (CFL step)
template <int EQ, int D>
__global__ void __launch_bounds__(NTHREADS) k_wave(Grid g, int l)
{
    pdl_enter();
    constexpr int M = EQ == 2 ? D + 2 : 1;
    const int cnt = g.counts[l];
    const int* list = g.leaves + g.off[l];
    const long long N = g.N[l];
    double w = 0.0;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += gridDim.x * blockDim.x) {
        const long long id = list[t];
        if (id < 0 || id >= N) continue;
        const double* qe = fbase(g, F_QE, l) + id;
        double q[M];
#pragma unroll
        for (int v = 0; v < M; ++v) q[v] = qe[v * N];
        const double s = wave_speed<EQ, D, M>(g, q);
        w = fmax(w, s != s ? 1e300 : s);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w = fmax(w, __shfl_xor_sync(0xffffffffu, w, o));
    if ((threadIdx.x & 31) == 0 && w > 0.0)
        atomicMax(g.wmax, (unsigned long long)__double_as_longlong(w));
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

void launch_wave(const Grid& g, cudaStream_t st, int l)
{
#define MRLT_CASE(E, DD)                                          \
    if (g.eq == E && g.d == DD) {                                 \
        k_wave<E, DD><<<grid_for(g, l), NTHREADS, 0, st>>>(g, l); \
        return;                                                   \
    }
    MRLT_CASE(0, 1) MRLT_CASE(0, 2) MRLT_CASE(0, 3)
    MRLT_CASE(1, 1) MRLT_CASE(1, 2) MRLT_CASE(1, 3)
    MRLT_CASE(2, 1) MRLT_CASE(2, 2) MRLT_CASE(2, 3)
    MRLT_CASE(3, 1) MRLT_CASE(3, 2) MRLT_CASE(3, 3)
#undef MRLT_CASE
}

} // namespace mrlt

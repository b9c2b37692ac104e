// mrlt_macro_eq.cu -- instantiates the persistent macro-step kernels of one
// equation, selected by MRLT_STAGE_EQ (0 advection, 1 Burgers, 2 Euler, 3
// reaction-diffusion) at compile time, for d = 1, 2, 3 and both flux
// precisions; a translation unit of its own so that it compiles in parallel
// with the stage kernels.
#include "mrlt_macro.cuh"

#ifndef MRLT_STAGE_EQ
#error "compile with -DMRLT_STAGE_EQ=<equation id>"
#endif

namespace mrlt {

template <>
int launch_macro_eq<MRLT_STAGE_EQ>(const Grid& g, cudaStream_t st, const MacroArgs* a)
{
    constexpr int E = MRLT_STAGE_EQ;
    switch (g.d) {
    case 1: return g.prec ? macro_dispatch<E, 1, float>(g, st, a) : macro_dispatch<E, 1, double>(g, st, a);
    case 2: return g.prec ? macro_dispatch<E, 2, float>(g, st, a) : macro_dispatch<E, 2, double>(g, st, a);
    case 3: return g.prec ? macro_dispatch<E, 3, float>(g, st, a) : macro_dispatch<E, 3, double>(g, st, a);
    default: return -1;
    }
}

} // namespace mrlt

// mrlt_stage_eq.cu -- instantiates the stage kernels of one equation,
// selected by MRLT_STAGE_EQ (0 advection, 1 Burgers, 2 Euler, 3 reaction-
// diffusion) at compile time, for d = 1, 2, 3 and both flux precisions.
#include "mrlt_stage.cuh"

#ifndef MRLT_STAGE_EQ
#error "compile with -DMRLT_STAGE_EQ=<equation id>"
#endif

namespace mrlt {

template <>
int launch_stage_eq<MRLT_STAGE_EQ>(const Grid& g, cudaStream_t st, int lo, int hi, int s, int lmin, double b,
                                   int reg)
{
    constexpr int E = MRLT_STAGE_EQ;
    switch (g.d) {
    case 1:
        return g.prec ? stage_dispatch<E, 1, float>(g, st, lo, hi, s, lmin, b, reg)
                      : stage_dispatch<E, 1, double>(g, st, lo, hi, s, lmin, b, reg);
    case 2:
        return g.prec ? stage_dispatch<E, 2, float>(g, st, lo, hi, s, lmin, b, reg)
                      : stage_dispatch<E, 2, double>(g, st, lo, hi, s, lmin, b, reg);
    case 3:
        return g.prec ? stage_dispatch<E, 3, float>(g, st, lo, hi, s, lmin, b, reg)
                      : stage_dispatch<E, 3, double>(g, st, lo, hi, s, lmin, b, reg);
    default:
        return 0;
    }
}

} // namespace mrlt

/*
 * mr_oracle.h -- plain, slow FP64 CPU oracle of adaptive cell-average
 * multiresolution (MR) with local time-stepping by natural continuous
 * extension of Runge-Kutta (MRLT/NERK), Lopes, Domingues, Schneider, Mendes,
 * "Local time-stepping for adaptive multiresolution using natural extension
 * of Runge-Kutta methods" (arXiv 1905.08717).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the parity reference for the
 * CUDA path.  It shares no code, header, table or helper with the CUDA
 * library, and nothing in the product imports it; only the tests, the
 * smoke check and the benchmark's CPU-baseline leg load it.
 *
 * Calls mirror the CUDA library's C-ABI so tests can drive both the same
 * way; all buffers are host memory owned by the caller.
 */
#ifndef MR_ORACLE_H
#define MR_ORACLE_H
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct or_config {
    int    dim;         /* 1, 2 or 3 space dimensions (Eq. 1)                 */
    int    equation;    /* 0 advection, 1 Burgers, 2 Euler, 3 reaction-diff.  */
    int    max_level;   /* L, finest level                                    */
    int    min_level;   /* coarsest leaf level; macro step = 2^(L-min) iters */
    double eps;         /* threshold epsilon (Alg. 2); 0 => no coarsening     */
    int    eps_mode;    /* 0 fixed eps, 1 level-scaled eps_l = 2^{d(l-L)} eps */
    int    rk_order;    /* 2 or 3 (Sec. 3, compact formulation)               */
    int    time_mode;   /* 0 global time step (MR/RK), 1 MRLT/NERK            */
    int    precision;   /* must be 0 (FP64)                                   */
    int    adapt_mode;  /* 0 fixed tree, 1 at macro-step start, 2 every LT iteration */
    int    reflux;      /* 1: conservative flux registers at coarse-fine faces */
    double cfl;         /* Courant number sigma                               */
    double lo[3], hi[3];/* box                                                */
    int    bc[3];       /* 0 periodic, 1 homogeneous Neumann (even mirror),
                           2 zero Dirichlet (odd mirror; scalar equations)    */
    double phys[8];     /* advection: a_x,a_y,a_z | Euler: gamma | RD: D,k,a  */
    int    flux;        /* 0: the equation's default flux (Euler: HLL);
                           1: AUSM+ (Euler only), the paper's flux (Sec. 5)   */
} or_config;

enum { OR_OK = 0, OR_E_INVALID = 1, OR_E_NOMEM = 2, OR_E_STATE = 5, OR_E_NUMERIC = 6 };

enum {
    OR_READ_LEAF_KEYS = 0,   /* int32 [n_leaves][4]: level, i, j, k            */
    OR_READ_LEAF_VALUES = 1, /* double [n_leaves][m] (level-major, then cell)  */
    OR_READ_UNIFORM = 2,     /* double [m][2^{dL}]: inverse MR transform to L  */
    OR_READ_STATS = 3,       /* double [64], see or_stats layout in the .c     */
    OR_READ_FIELDS = 4,      /* double [n_leaves][8][m]: q^n q* q** q^{n+1}
                                NERK(1/2) NERK(1/4) NERK(3/4) Eq.14 value      */
    OR_READ_NODES = 5        /* double [n_internal][4 + 7 m]: level, i, j, k, then
                                q^n, q*, q**, q^{n+1}, half-step value (Eq. 17),
                                theta=1/4 (Alg. 9), theta=3/4 (Eq. 20) as stored
                                by the latest iteration                        */
};

int  or_create(const or_config* cfg, const double* q0_finest, void** out);
int  or_set_tree(void* h, const unsigned char* leaf_level_finest);
int  or_adapt(void* h);
int  or_step(void* h, double t_target, long long* iters_out);
int  or_iterate(void* h, double dt, long long n_iters, long long* iters_out);
int  or_read(void* h, int what, void* buf, size_t cap_bytes, size_t* used);
void or_destroy(void* h);
const char* or_last_error(void* h);

/* Numerical flux of the configured equation across the face between cells 1
 * and 2 of the 4-cell stencil W (conservative values, [cell][variable]) in
 * direction k, face width dxf: the function the solver uses, exported for
 * tests.  Returns OR_E_INVALID for a bad configuration. */
int or_num_flux(const or_config* cfg, int k, double dxf, const double* W, double* F);

#ifdef __cplusplus
}
#endif
#endif

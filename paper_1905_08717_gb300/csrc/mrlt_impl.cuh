// mrlt_impl.cuh -- device data layout and shared device routines of the
// MRLT/NERK library (private to the library; the public C-ABI is mrlt.h).
//
// Data layout in HBM (one solver instance):
//   every level l in [min_level, L] indexes its N_l = 2^{d l} cells as
//   id = i + n_l (j + n_l k), n_l = 2^l; the per-cell maps of all levels live
//   in one "pyramid" allocation at offset off[l] (cells):
//   - status (uint8): 0 absent, 1 leaf, 2 internal node; refinement flags (uint8)
//   - slot (int32): the node's slot in the node arrays, -1 when absent
//   The values live only where nodes exist: node arrays of `cap` slots, each
//   node's m variables contiguous ([slot][v]); slot 0 is a sink that never
//   belongs to a node (see the capacity rule in mrlt_api.cu):
//   - fields, float64, or float32 in the mixed-precision mode (the state is
//     stored, and the stage arithmetic done, in FP32; registers and the detail
//     test stay FP64):
//       Q0 q^n, Q1 q*, Q2 q**, QE q^{n+1} (leaves: compact RK stages of Sec. 3;
//       internal nodes: the projections / refreshed values of Algs. 3-9),
//       XH half-step value (Eq. 17), NH, N1, N3 the NERK theta = 1/2, 1/4, 3/4
//       values of internal nodes.  Leaves never store NERK values: they are
//       recomputed from Q0, Q1, Q2, QE where needed (same polynomial).
//   - registers (float64, [slot][face][v]): the time-integrated flux through
//       each face of a leaf whose neighbour across it is on another level (a
//       coarse leaf at a face to finer nodes, or a fine leaf at a face to a
//       coarser leaf).  One array serves both roles: the kind of a face cannot
//       change while its register holds a value (the restricted remesh keeps
//       both sides until the coarse step ends, when the reflux clears them).
//   - per-level compact lists (int32) of leaves and internal nodes, ascending
//     cell id, rebuilt after every remesh by warp-ballot stream compaction.
//   Free slots form a stack (fstack, ftop[0] entries); a remesh releases the
//   slots of removed nodes, then pops slots for new nodes (ftop[1] counts the
//   pops until the next compaction commits them).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace mrlt {

constexpr int LMAX = 16;
constexpr int MMAX = 5;
constexpr int NTHREADS = 128;
// tiles of the tiled stage kernel (d = 1: 64 cells; d = 2: 16 x 8; d = 3: 8 x 4 x 4)
constexpr int kTile1X = 64;
constexpr int kTile2X = 16, kTile2Y = 8;
constexpr int kTile3X = 8, kTile3Y = 4, kTile3Z = 4;
// threads per tile CTA: two per cell (measured: 3D blast L=8 -10 to -13%, 2D
// Euler L=10 -1.5% against one per cell; four per cell was slower)
constexpr int kTileThreads1 = 128, kTileThreads2 = 256, kTileThreads3 = 256;

enum Field { F_Q0 = 0, F_Q1, F_Q2, F_QE, F_XH, F_NH, F_N1, F_N3, NFIELD };
enum Kind { K_WALL = 0, K_LEAF = 1, K_FINER = 2, K_COARSER = 3 };
enum FlagBits { FL_SIG = 1, FL_BIG = 2, FL_DES = 4, FL_ALLOW = 8, FL_REF = 16 };
enum ErrBits { ERR_INDEX = 1, ERR_SOURCE = 2, ERR_NONFINITE = 4, ERR_REFLUX = 8, ERR_TIMEOUT = 16, ERR_CAPACITY = 32 };

struct Grid {
    uint8_t* st;
    uint8_t* flag;
    int* slot;                      // per cell: node slot, -1 when absent
    int* fstack;                    // free slots
    int* ftop;                      // [0] free slots on the stack, [1] pops not yet committed
    long long cap;                  // node slots (slot 0 is the sink)
    void* f[NFIELD];                // node fields: double, or float when prec = 1
    double* rg;                     // flux registers of the nodes, [slot][face][v]
    int* leaves;
    int* inner;
    int* counts;                    // [0..LMAX] leaves, [LMAX+1..] internal nodes, [2(LMAX+1)..] active tiles
    uint8_t* tflag;                 // per-level tile flags (tile holds a leaf)
    int* tlist;                     // per-level lists of active tiles, ascending
    double* scale;                  // [MMAX] detail normalisation s_v
    unsigned long long* scale_bits; // [MMAX] running max |q_v| (bit pattern)
    int* err;
    unsigned long long* near;
    unsigned long long* wmax;
    unsigned long long* updates;
    unsigned long long* work;       // [(LMAX+1) * 4]: leaf-stages per level and stage
    double* dtp;                    // fine step dt of the current macro step (device scalar)
    int* room;                      // [0] refinement flags being counted, [1] halt: iteration + 1, [2] nodes needed
    long long off[LMAX + 1];
    long long N[LMAX + 1];
    int n[LMAX + 1];
    double dx[LMAX + 1][3];
    double rdx[LMAX + 1][3];        // 1 / dx
    long long toff[LMAX + 1];       // tile offset of each level in tflag / tlist
    int ntx[LMAX + 1], nty[LMAX + 1], ntz[LMAX + 1]; // tiles per direction
    int d, m, nf, L, lb, eq, rk, gts;
    int bc[3];
    double phys[8];
    double eps;
    int eps_mode;
    int prec;                       // 0 FP64, 1 mixed: state, fluxes and stage updates in FP32
    int flux;                       // Euler: 0 HLL, 1 AUSM+
    double igm;                     // Euler: 1 / (gamma - 1)
    int gcap;                       // CTAs per stage launch at most (0: resident capacity)
};

// Programmatic dependent launch (sm_90 and later).  Every kernel starts by
// waiting until the kernel before it in the stream has completed and its
// writes are visible (griddepcontrol.wait), then allows the next kernel's
// launch to begin (griddepcontrol.launch_dependents).  The launch and the CTA
// setup of the next kernel thus overlap the tail of this one.  Both are no-ops
// in a kernel launched without a programmatic dependency.
__device__ __forceinline__ void pdl_enter()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// A remesh inside a macro step whose new tree would need more node slots than
// the arrays hold halts the solver's device work (room[1] != 0): every later
// kernel of the fine iterations returns at its start, until the host has
// grown the arrays, cleared the halt and resumed at the halted iteration.
// Read after pdl_enter, so that a halt set by an earlier kernel is visible.
__device__ __forceinline__ bool halted(const Grid& g) { return g.room[1] != 0; }

#define MRLT_ENTER(g)         \
    do {                      \
        pdl_enter();          \
        if (halted(g)) return; \
    } while (0)

// Launch with programmatic stream serialisation: the kernel may be launched
// before its predecessor in the stream has finished; it waits in pdl_enter().
template <class... KArgs, class... Args>
inline cudaError_t pdl_launch(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, args...);
}

// exposure context: level u being updated, stage s (0 = plain q^n), lmin
struct Ctx {
    int u, s, lmin;
};

// Ghost rule, the same on every level: periodic wrap; homogeneous Neumann as
// an even mirror; zero Dirichlet (scalar equations) as an odd mirror, the
// ghost taking the negated value: the parity neg flips at every reflection
// on a Dirichlet wall (an odd count negates the value).
__device__ __forceinline__ int wrap_or_mirror(const Grid& g, int l, int k, int p, int& neg)
{
    const int n = g.n[l];
    if (g.bc[k] == 0) return p & (n - 1); // periodic wrap (n = 2^l)
    const int odd = g.bc[k] == 2;
#pragma unroll 1
    for (int it = 0; it < 8 && (p < 0 || p >= n); ++it) {
        p = p < 0 ? -1 - p : 2 * n - 1 - p;
        neg ^= odd;
    }
    return p < 0 ? 0 : (p >= n ? n - 1 : p);
}

// neighbourhood rule of the tree: wrap when periodic, drop cells past a wall
__device__ __forceinline__ bool in_box(const Grid& g, int l, int k, int p, int* q)
{
    const int n = g.n[l];
    if (g.bc[k] == 0) {
        *q = p & (n - 1); // periodic wrap (n = 2^l)
        return true;
    }
    if (p < 0 || p >= n) return false;
    *q = p;
    return true;
}

__device__ __forceinline__ long long cell_id(const Grid& g, int l, int x, int y, int z)
{
    const long long n = g.n[l];
    return (long long)x + n * ((long long)y + n * (long long)z);
}

// coordinates of cell id on level l (n = 2^l cells per direction)
__device__ __forceinline__ void cell_xyz(const Grid& g, int l, long long id, int c[3])
{
    const long long mask = (1LL << l) - 1;
    c[0] = (int)(id & mask);
    c[1] = g.d > 1 ? (int)((id >> l) & mask) : 0;
    c[2] = g.d > 2 ? (int)(id >> (2 * l)) : 0;
}

// the m values of field f of the node in slot sl, stored as T (double, or
// float in the mixed mode); a negative slot (an absent cell) reads the sink
template <class T>
__device__ __forceinline__ T* nd(const Grid& g, int f, int sl)
{
    return static_cast<T*>(g.f[f]) + (long long)(sl < 0 ? 0 : sl) * g.m;
}

__device__ __forceinline__ int slot_of(const Grid& g, int l, long long id)
{
    return g.slot[g.off[l] + id];
}

// registers of the node in slot sl: [face][v]
__device__ __forceinline__ double* regs(double* r, const Grid& g, int sl)
{
    return r + (long long)(sl < 0 ? 0 : sl) * g.nf * g.m;
}

__device__ __forceinline__ uint8_t status(const Grid& g, int l, long long id)
{
    return g.st[g.off[l] + id];
}

// Value of the stored node of level l in slot sl (status st) as seen by the stencil of a
// level-u leaf at stage x.s of the current iteration: the exposure table of
// Secs. 4.1-4.3 / Algs. 3-9.  Leaves recompute their NERK values from the
// stage values: with k1 = q* - q^n and k2 the second stage increment
// (RK2: k2 = 2 q^{n+1} - q^n - q*, RK3: k2 = 4 q** - 3 q^n - q*),
// q(theta) = q^n + (theta - theta^2/2) k1 + theta^2/2 k2 (Sec. 3 NERK2).
// T is the storage type of the fields, O the arithmetic type of the result.
template <int M, class T, class O>
__device__ __forceinline__ void expose(const Grid& g, const Ctx& x, int l, int sl, int st, O* out)
{
    const T* q0 = nd<T>(g, F_Q0, sl);
    const T* q1 = nd<T>(g, F_Q1, sl);
    const T* q2 = nd<T>(g, F_Q2, sl);
    const T* qe = nd<T>(g, F_QE, sl);
    const int s = x.s;
    const int rel = l - x.u;
    if (s == 0 || (s == 1 && g.gts) || (s == 1 && (rel >= 0 || l >= x.lmin))) {
#pragma unroll
        for (int v = 0; v < M; ++v) out[v] = O(q0[v]);
        return;
    }
    if (g.gts) {
        const T* a = s == 2 ? q1 : q2;
#pragma unroll
        for (int v = 0; v < M; ++v) out[v] = O(a[v]);
        return;
    }
    if (s == 1) { // coarser level lmin-1, mid-step: theta = 1/2 value
        if (g.rk == 3) {
#pragma unroll
            for (int v = 0; v < M; ++v) out[v] = O(q2[v]);
        } else if (st == 1) {
#pragma unroll
            for (int v = 0; v < M; ++v)
                out[v] = O(0.5) * O(q0[v]) + O(0.25) * O(q1[v]) + O(0.25) * O(qe[v]);
        } else {
            const T* nh = nd<T>(g, F_NH, sl);
#pragma unroll
            for (int v = 0; v < M; ++v) out[v] = O(nh[v]);
        }
        return;
    }
    if (s == 2) {
        if (rel == 0) {
#pragma unroll
            for (int v = 0; v < M; ++v) out[v] = O(q1[v]);
        } else if (rel == 1) {
            if (st == 1) { // Eq. 14: q* + k2
                if (g.rk == 2) {
#pragma unroll
                    for (int v = 0; v < M; ++v) out[v] = O(2) * O(qe[v]) - O(q0[v]);
                } else {
#pragma unroll
                    for (int v = 0; v < M; ++v) out[v] = O(4) * O(q2[v]) - O(3) * O(q0[v]);
                }
            } else { // Eq. 15
#pragma unroll
                for (int v = 0; v < M; ++v) out[v] = O(2) * O(q1[v]) - O(q0[v]);
            }
        } else if (l >= x.lmin) { // half step of the coarser level
            if (st == 1) {
#pragma unroll
                for (int v = 0; v < M; ++v) out[v] = O(q0[v]) + O(0.5) * (O(q1[v]) - O(q0[v]));
            } else {
                const T* xh = nd<T>(g, F_XH, sl);
#pragma unroll
                for (int v = 0; v < M; ++v) out[v] = O(xh[v]);
            }
        } else { // end of the mid-step coarser level
#pragma unroll
            for (int v = 0; v < M; ++v) out[v] = O(qe[v]);
        }
        return;
    }
    // stage 3
    if (rel == 0) {
#pragma unroll
        for (int v = 0; v < M; ++v) out[v] = O(q2[v]);
    } else if (rel == 1) {
#pragma unroll
        for (int v = 0; v < M; ++v) out[v] = O(qe[v]);
    } else {
        const bool act = l >= x.lmin;
        if (st == 1) {
            const O b1 = act ? O(7.0 / 32.0) : O(15.0 / 32.0);
            const O b2 = act ? O(1.0 / 32.0) : O(9.0 / 32.0);
#pragma unroll
            for (int v = 0; v < M; ++v) {
                const O a0 = O(q0[v]), a1 = O(q1[v]);
                const O k1 = a1 - a0;
                const O k2 = O(4) * O(q2[v]) - O(3) * a0 - a1;
                out[v] = a0 + b1 * k1 + b2 * k2;
            }
        } else {
            const T* nn = nd<T>(g, act ? F_N1 : F_N3, sl);
#pragma unroll
            for (int v = 0; v < M; ++v) out[v] = O(nn[v]);
        }
    }
}

// 1D prediction weights of Eq. 4 for child offset a (0 left, 1 right):
// child = parent + s (right - left) / 8, s = -1 for a = 0, +1 for a = 1.
__device__ __forceinline__ double pw(int a, int delta)
{
    if (delta == 0) return 1.0;
    const double s = a ? 0.125 : -0.125;
    return delta > 0 ? s : -s;
}

// Tensor-product prediction (Eq. 4 applied along each direction) of the cell
// at in-box coordinates q of level l from the 3^d stored nodes of level l-1
// around its parent, using their exposures.
template <int D, int M, class T, class O>
__device__ __forceinline__ void predict(const Grid& g, const Ctx& x, int l, const int q[3], O* out)
{
    const int pl = l - 1;
#pragma unroll
    for (int v = 0; v < M; ++v) out[v] = O(0);
    if (pl < g.lb) {
        atomicOr(g.err, ERR_SOURCE);
        return;
    }
    const int P0 = q[0] >> 1, P1 = q[1] >> 1, P2 = q[2] >> 1;
    const int a0 = q[0] & 1, a1 = q[1] & 1, a2 = q[2] & 1;
    // in 3D the outer loops stay rolled: 27 inlined exposures per prediction
    // site cost far more compile time than the loop overhead they save
#pragma unroll(D > 2 ? 1 : 3)
    for (int dz = (D > 2 ? -1 : 0); dz <= (D > 2 ? 1 : 0); ++dz) {
        int nz = 0;
        const int z = D > 2 ? wrap_or_mirror(g, pl, 2, P2 + dz, nz) : 0;
        const O wz = D > 2 ? O(pw(a2, dz)) : O(1);
#pragma unroll(D > 2 ? 1 : 3)
        for (int dy = (D > 1 ? -1 : 0); dy <= (D > 1 ? 1 : 0); ++dy) {
            int nyz = nz;
            const int y = D > 1 ? wrap_or_mirror(g, pl, 1, P1 + dy, nyz) : 0;
            const O wyz = wz * (D > 1 ? O(pw(a1, dy)) : O(1));
#pragma unroll
            for (int dxx = -1; dxx <= 1; ++dxx) {
                int neg = nyz;
                const int xx = wrap_or_mirror(g, pl, 0, P0 + dxx, neg);
                const long long id = cell_id(g, pl, xx, y, z);
                const int st = status(g, pl, id);
                const int sl = slot_of(g, pl, id);
                if (st == 0) {
                    atomicOr(g.err, ERR_SOURCE);
                    continue;
                }
                O val[M];
                expose<M, T, O>(g, x, pl, sl, st, val);
                const O w0 = wyz * O(pw(a0, dxx));
                const O w = neg ? -w0 : w0; // an odd-mirror ghost enters negated
#pragma unroll
                for (int v = 0; v < M; ++v) out[v] += w * val[v];
            }
        }
    }
}

// Predictions (Eq. 4, tensor product) of all 2^d children on level l + 1 of
// the node at in-box coordinates c of level l: the 3^d block around c is read
// once and enters every child with that child's weights.  Each child's sum
// runs over the block in the order of predict(), so out[k] equals
// predict(g, x, l + 1, 2 c + k) term by term.
template <int D, int M, class T>
__device__ __forceinline__ void predict_children(const Grid& g, const Ctx& x, int l, const int c[3],
                                                 double (*out)[M])
{
    constexpr int NCH = 1 << D;
#pragma unroll
    for (int k = 0; k < NCH; ++k)
#pragma unroll
        for (int v = 0; v < M; ++v) out[k][v] = 0.0;
#pragma unroll(D > 2 ? 1 : 3)
    for (int dz = (D > 2 ? -1 : 0); dz <= (D > 2 ? 1 : 0); ++dz) {
        int nz = 0;
        const int z = D > 2 ? wrap_or_mirror(g, l, 2, c[2] + dz, nz) : 0;
#pragma unroll(D > 2 ? 1 : 3)
        for (int dy = (D > 1 ? -1 : 0); dy <= (D > 1 ? 1 : 0); ++dy) {
            int nyz = nz;
            const int y = D > 1 ? wrap_or_mirror(g, l, 1, c[1] + dy, nyz) : 0;
#pragma unroll
            for (int dxx = -1; dxx <= 1; ++dxx) {
                int neg = nyz;
                const int xx = wrap_or_mirror(g, l, 0, c[0] + dxx, neg);
                const long long id = cell_id(g, l, xx, y, z);
                const int st = status(g, l, id);
                const int sl = slot_of(g, l, id);
                if (st == 0) {
                    atomicOr(g.err, ERR_SOURCE);
                    continue;
                }
                double val[M];
                expose<M, T, double>(g, x, l, sl, st, val);
#pragma unroll
                for (int k = 0; k < NCH; ++k) {
                    const double wz = D > 2 ? pw((k >> 2) & 1, dz) : 1.0;
                    const double wyz = wz * (D > 1 ? pw((k >> 1) & 1, dy) : 1.0);
                    const double w0 = wyz * pw(k & 1, dxx);
                    const double w = neg ? -w0 : w0; // an odd-mirror ghost enters negated
#pragma unroll
                    for (int v = 0; v < M; ++v) out[k][v] += w * val[v];
                }
            }
        }
    }
}

// value of the cell at (possibly out-of-box) coordinates p on level l
template <int D, int M, class T, class O>
__device__ __forceinline__ void value_at(const Grid& g, const Ctx& x, int l, const int p[3], O* out)
{
    int q[3] = {0, 0, 0};
    int neg = 0;
#pragma unroll
    for (int k = 0; k < D; ++k) q[k] = wrap_or_mirror(g, l, k, p[k], neg);
    const long long id = cell_id(g, l, q[0], q[1], q[2]);
    const int st = status(g, l, id);
    if (st) expose<M, T, O>(g, x, l, slot_of(g, l, id), st, out);
    else predict<D, M, T, O>(g, x, l, q, out);
    if (neg) {
#pragma unroll
        for (int v = 0; v < M; ++v) out[v] = -out[v];
    }
}

// ---------------------------------------------------------------- physics
template <class R>
__device__ __forceinline__ R minmod(R a, R b)
{
    if (a * b <= R(0)) return R(0);
    return fabs(a) < fabs(b) ? a : b;
}

// Variables that MUSCL reconstructs: primitives (rho, u_1..u_d, p) for Euler,
// the conserved variable itself otherwise.  R is the arithmetic type of the
// flux evaluation: double, or float in the mixed-precision mode; W holds the
// conservative values (type WT).
template <int EQ, int D, int M, class R, class WT>
__device__ __forceinline__ void recon_vars(const Grid& g, const WT* W, R* P)
{
    if constexpr (EQ == 2) {
        const R gam = R(g.phys[0]);
        const R rho = R(W[0]);
        const R ir = R(1) / rho;
        R ke = R(0);
        P[0] = rho;
#pragma unroll
        for (int c = 0; c < D; ++c) {
            P[1 + c] = R(W[1 + c]) * ir;
            ke += R(W[1 + c]) * P[1 + c];
        }
        P[D + 1] = (gam - R(1)) * (R(W[D + 1]) - R(0.5) * ke);
    } else {
#pragma unroll
        for (int v = 0; v < M; ++v) P[v] = R(W[v]);
    }
}

// AUSM+ (Liou 1996), the paper's Euler flux (Sec. 5), across a face normal
// to direction k, from the reconstructed primitives (rho, u_1..u_d, p) and
// conservative states of both sides.  With total enthalpy H = (E + p)/rho
// and critical speed a*^2 = 2 (g-1)/(g+1) H, the interface speed is
// a = min(a*_L^2 / max(a*_L, u_L), a*_R^2 / max(a*_R, -u_R)); the Mach
// numbers M = u/a are split as M+-(M) = +-(M +- 1)^2/4 +- (M^2 - 1)^2/8 and
// pressure as P+-(M) = (M +- 1)^2 (2 -+ M)/4 +- 3/16 M (M^2 - 1)^2 when
// |M| < 1 (upwind values otherwise); the flux is
// a (max(m, 0) Psi_L + min(m, 0) Psi_R) + p_half e_k, Psi = rho (1, u, H),
// m = M+(M_L) + M-(M_R), p_half = P+(M_L) p_L + P-(M_R) p_R.
template <class R>
__device__ __forceinline__ R ausm_split_mach(R M, R sgn)
{
    if (fabs(M) >= R(1)) return R(0.5) * (M + sgn * fabs(M));
    const R t = M * M - R(1);
    return sgn * R(0.25) * (M + sgn) * (M + sgn) + sgn * R(0.125) * t * t;
}

template <class R>
__device__ __forceinline__ R ausm_split_pres(R M, R sgn)
{
    if (fabs(M) >= R(1)) return M * sgn > R(0) ? R(1) : R(0);
    const R t = M * M - R(1);
    return R(0.25) * (M + sgn) * (M + sgn) * (R(2) - sgn * M) + sgn * R(0.1875) * M * t * t;
}

template <int D, int M, class R>
__device__ __forceinline__ void ausm_plus(R gam, int k, const R* PL, const R* PR, const R* UL, const R* UR, R* F)
{
    const R pL = PL[D + 1], pR = PR[D + 1];
    const R HL = (UL[D + 1] + pL) / PL[0], HR = (UR[D + 1] + pR) / PR[0];
    const R uL = PL[1 + k], uR = PR[1 + k];
    const R cst = R(2) * (gam - R(1)) / (gam + R(1));
    const R asL = sqrt(cst * HL), asR = sqrt(cst * HR);
    const R atL = asL * asL / fmax(asL, uL);
    const R atR = asR * asR / fmax(asR, -uR);
    const R a = fmin(atL, atR);
    const R ML = uL / a, MR = uR / a;
    const R mh = ausm_split_mach(ML, R(1)) + ausm_split_mach(MR, R(-1));
    const R ph = ausm_split_pres(ML, R(1)) * pL + ausm_split_pres(MR, R(-1)) * pR;
    const R mp = fmax(mh, R(0)), mm = fmin(mh, R(0));
    F[0] = a * (mp * PL[0] + mm * PR[0]);
#pragma unroll
    for (int c = 0; c < D; ++c) F[1 + c] = a * (mp * UL[1 + c] + mm * UR[1 + c]);
    F[D + 1] = a * (mp * (PL[0] * HL) + mm * (PR[0] * HR));
    F[1 + k] += ph;
}

// Numerical flux along direction k across the face between stencil cells 1
// and 2 of a 4-cell stencil, from their reconstruction variables P(i, v).
template <int EQ, int D, int M, class R, class Acc>
__device__ __forceinline__ void flux_recon(const Grid& g, int k, double dxf, const Acc& P, R* F)
{
    const R h = R(0.5);
    if constexpr (EQ == 0) { // linear advection, centred flux
        F[0] = R(g.phys[k]) * (P(1, 0) + P(2, 0)) * h;
    } else if constexpr (EQ == 3) { // two-point diffusive flux
        F[0] = -R(g.phys[0]) * (P(2, 0) - P(1, 0)) / R(dxf);
    } else if constexpr (EQ == 1) { // Burgers: MUSCL-minmod + Godunov
        const R u0 = P(0, 0), u1 = P(1, 0), u2 = P(2, 0), u3 = P(3, 0);
        const R uL = u1 + h * minmod(u1 - u0, u2 - u1);
        const R uR = u2 - h * minmod(u2 - u1, u3 - u2);
        const R fL = h * uL * uL, fR = h * uR * uR;
        if (uL <= uR) F[0] = uL > R(0) ? fL : (uR < R(0) ? fR : R(0));
        else F[0] = fmax(fL, fR);
    } else { // Euler: MUSCL-minmod on (rho, u_1..u_d, p) + HLL
        const R gam = R(g.phys[0]);
        R PL[M], PR[M];
#pragma unroll
        for (int v = 0; v < M; ++v) {
            const R a0 = P(0, v), a1 = P(1, v), a2 = P(2, v), a3 = P(3, v);
            PL[v] = a1 + h * minmod(a1 - a0, a2 - a1);
            PR[v] = a2 - h * minmod(a2 - a1, a3 - a2);
        }
        R UL[M], UR[M], FL[M], FR[M];
        R keL = R(0), keR = R(0);
        UL[0] = PL[0];
        UR[0] = PR[0];
#pragma unroll
        for (int c = 0; c < D; ++c) {
            UL[1 + c] = PL[0] * PL[1 + c];
            UR[1 + c] = PR[0] * PR[1 + c];
            keL += PL[1 + c] * PL[1 + c];
            keR += PR[1 + c] * PR[1 + c];
        }
        const R igm = R(g.igm);
        UL[D + 1] = PL[D + 1] * igm + h * PL[0] * keL;
        UR[D + 1] = PR[D + 1] * igm + h * PR[0] * keR;
        const R unL = PL[1 + k], unR = PR[1 + k];
        if (g.flux == 1) { // AUSM+
            ausm_plus<D, M, R>(gam, k, PL, PR, UL, UR, F);
            return;
        }
#pragma unroll
        for (int v = 0; v < M; ++v) {
            FL[v] = UL[v] * unL;
            FR[v] = UR[v] * unR;
        }
        FL[1 + k] += PL[D + 1];
        FR[1 + k] += PR[D + 1];
        FL[D + 1] += PL[D + 1] * unL;
        FR[D + 1] += PR[D + 1] * unR;
        // sound speeds sqrt(gamma p / rho) = gamma p rsqrt(gamma p rho)
        const R gpL = gam * PL[D + 1], gpR = gam * PR[D + 1];
        const R cL = gpL * rsqrt(gpL * PL[0]);
        const R cR = gpR * rsqrt(gpR * PR[0]);
        const R sL = fmin(unL - cL, unR - cR);
        const R sR = fmax(unL + cL, unR + cR);
        if (sL >= R(0)) {
#pragma unroll
            for (int v = 0; v < M; ++v) F[v] = FL[v];
        } else if (sR <= R(0)) {
#pragma unroll
            for (int v = 0; v < M; ++v) F[v] = FR[v];
        } else {
            const R ids = R(1) / (sR - sL);
#pragma unroll
            for (int v = 0; v < M; ++v) F[v] = (sR * FL[v] - sL * FR[v] + sL * sR * (UR[v] - UL[v])) * ids;
        }
    }
}

template <int EQ, int M, class R>
__device__ __forceinline__ void source(const Grid& g, const R* q, R* S)
{
#pragma unroll
    for (int v = 0; v < M; ++v) S[v] = R(0);
    if constexpr (EQ == 3) {
        const R u = q[0];
        S[0] = R(g.phys[1]) * u * (R(1) - u) * (u - R(g.phys[2]));
    }
}

template <int EQ, int D, int M>
__device__ __forceinline__ double wave_speed(const Grid& g, const double* q)
{
    double s = 0.0;
    if constexpr (EQ == 0) {
#pragma unroll
        for (int k = 0; k < D; ++k) s += fabs(g.phys[k]);
    } else if constexpr (EQ == 1) {
        s = D * fabs(q[0]);
    } else if constexpr (EQ == 2) {
        const double gam = g.phys[0], rho = q[0];
        double ke = 0.0;
#pragma unroll
        for (int k = 0; k < D; ++k) ke += q[1 + k] * q[1 + k] / rho;
        const double p = (gam - 1.0) * (q[D + 1] - 0.5 * ke);
        const double c = sqrt(gam * p / rho);
#pragma unroll
        for (int k = 0; k < D; ++k) s += fabs(q[1 + k] / rho) + c;
    }
    return s;
}

// ---------------------------------------------------------------- host side
struct Launch; // fwd

// kernel launchers (defined in the .cu files), all on stream `st`
// one compact RK stage s on every leaf of the levels lo..hi (independent
// levels only), fine step dt = *g.dtp (level u steps dt, or 2^{L-u} dt in LT
// mode), RK weight b of the stage; returns the number of kernel launches issued
// (-1 when the kernel could not be set up).  lo > hi only sets the kernel up.
int launch_stage(const Grid& g, cudaStream_t st, int lo, int hi, int s, int lmin, double b, int reg);
void launch_wave(const Grid& g, cudaStream_t st, int l);
// one persistent macro-step kernel launch (mrlt_macro.cuh); a == nullptr sets
// the kernel up only.  Returns 1 when launched, 0 after set-up, -1 on failure.
struct MacroArgs;
int launch_macro(const Grid& g, cudaStream_t st, const MacroArgs* a);
// the bounded grid barrier with `missing` CTAs that never arrive (self-test)
int launch_grid_wait_test(cudaStream_t st, int ctas, int missing, unsigned long long limit_ns, unsigned* bar,
                          int* err);
} // namespace mrlt

// mrlt_stage.cu -- the per-leaf stage kernel of the MR/MRLT time evolution:
// face fluxes from the exposures of Secs. 4.1-4.3, the compact RK update of
// Sec. 3 and the flux-register epilogue.  One thread per leaf of one level.
#include "mrlt_impl.cuh"

namespace mrlt {

// Face flux of the leaf at c (level u) in direction k, side -1/+1, oriented
// along +x_k (Sec. 2 flux scenarios).  Returns the face kind.
template <int EQ, int D, int M>
__device__ __forceinline__ int face_flux(const Grid& g, const Ctx& x, int u, const int c[3], int k,
                                         int side, double* F)
{
    int kind, q;
    bool sub = false;
    if (!in_box(g, u, k, c[k] + side, &q)) {
        kind = K_WALL;
    } else {
        int nb[3] = {c[0], c[1], c[2]};
        nb[k] = q;
        const int s = status(g, u, cell_id(g, u, nb[0], nb[1], nb[2]));
        if (s == 2 && u < g.L) {
            sub = true;
            kind = K_FINER;
        } else {
            kind = s == 1 ? K_LEAF : K_COARSER;
        }
    }
    double W[4][M];
    if (!sub) {
        int p[3] = {c[0], c[1], c[2]};
        const int first = side > 0 ? c[k] - 1 : c[k] - 2;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            p[k] = first + i;
            value_at<D, M>(g, x, u, p, W[i]);
        }
        num_flux<EQ, D, M>(g, k, g.dx[u][k], W, F);
        return kind;
    }
    // internal neighbour: mean of the 2^{d-1} sub-face fluxes on level u+1
    constexpr int NT = 1 << (D - 1);
    double acc[M];
#pragma unroll
    for (int v = 0; v < M; ++v) acc[v] = 0.0;
#pragma unroll 1
    for (int t = 0; t < NT; ++t) {
        int p[3] = {0, 0, 0}, bit = 0;
#pragma unroll
        for (int j = 0; j < D; ++j) {
            if (j == k) continue;
            p[j] = 2 * c[j] + ((t >> bit) & 1);
            ++bit;
        }
        const int first = side > 0 ? 2 * c[k] : 2 * c[k] - 2;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            p[k] = first + i;
            value_at<D, M>(g, x, u + 1, p, W[i]);
        }
        double Fs[M];
        num_flux<EQ, D, M>(g, k, g.dx[u + 1][k], W, Fs);
#pragma unroll
        for (int v = 0; v < M; ++v) acc[v] += Fs[v];
    }
#pragma unroll
    for (int v = 0; v < M; ++v) F[v] = acc[v] * (1.0 / NT);
    return kind;
}

// One compact RK stage (Sec. 3) of every leaf of level u:
//   s = 1: q*  = q^n + dt_l f(q^n)
//   s = 2: RK2 q^{n+1} = q^n/2 + q*/2 + dt_l f(q*)/2 ; RK3 q** = 3q^n/4 + q*/4 + dt_l f(q*)/4
//   s = 3: q^{n+1} = q^n/3 + 2q**/3 + 2 dt_l f(q**)/3
// f from the exposures of stage s; registers get dt_l * b_s * F at coarse-fine faces.
template <int EQ, int D>
__global__ void __launch_bounds__(NTHREADS) k_stage(Grid g, int u, int s, int lmin, double dtl,
                                                    double bw, int reg)
{
    constexpr int M = EQ == 2 ? D + 2 : 1;
    const int cnt = g.counts[u];
    const int* list = g.leaves + g.off[u];
    const long long N = g.N[u];
    if (s == 1 && blockIdx.x == 0 && threadIdx.x == 0)
        atomicAdd(g.updates, (unsigned long long)cnt);
    const Ctx x{u, s, lmin};
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < cnt; t += gridDim.x * blockDim.x) {
        const long long id = list[t];
        if (id < 0 || id >= N) {
            atomicOr(g.err, ERR_INDEX);
            continue;
        }
        int c[3];
        cell_xyz(g, u, id, c);
        double self[M], f[M];
        expose<M>(g, x, u, id, 1, self);
        source<EQ, M>(g, self, f);
#pragma unroll 1
        for (int k = 0; k < D; ++k) {
            double Fm[M], Fp[M];
            const int km = face_flux<EQ, D, M>(g, x, u, c, k, -1, Fm);
            const int kp = face_flux<EQ, D, M>(g, x, u, c, k, +1, Fp);
            const double idx = 1.0 / g.dx[u][k];
#pragma unroll
            for (int v = 0; v < M; ++v) f[v] += (Fm[v] - Fp[v]) * idx;
            if (reg) {
                const long long roff = g.off[u] * g.nf * g.m;
                if (km == K_FINER || km == K_COARSER) {
                    double* R = (km == K_FINER ? g.rc : g.rf) + roff + id;
#pragma unroll
                    for (int v = 0; v < M; ++v) R[((2 * k) * M + v) * N] += bw * Fm[v];
                }
                if (kp == K_FINER || kp == K_COARSER) {
                    double* R = (kp == K_FINER ? g.rc : g.rf) + roff + id;
#pragma unroll
                    for (int v = 0; v < M; ++v) R[((2 * k + 1) * M + v) * N] += bw * Fp[v];
                }
            }
        }
        double* q0 = fbase_w(g, F_Q0, u) + id;
        double* q1 = fbase_w(g, F_Q1, u) + id;
        double* q2 = fbase_w(g, F_Q2, u) + id;
        double* qe = fbase_w(g, F_QE, u) + id;
#pragma unroll
        for (int v = 0; v < M; ++v) {
            const double kk = dtl * f[v];
            if (s == 1) {
                q1[v * N] = q0[v * N] + kk;
            } else if (s == 2) {
                if (g.rk == 2) qe[v * N] = 0.5 * q0[v * N] + 0.5 * q1[v * N] + 0.5 * kk;
                else q2[v * N] = 0.75 * q0[v * N] + 0.25 * q1[v * N] + 0.25 * kk;
            } else {
                qe[v * N] = (1.0 / 3.0) * q0[v * N] + (2.0 / 3.0) * q2[v * N] + (2.0 / 3.0) * kk;
            }
        }
    }
}

// largest sum of characteristic speeds over the leaves of level l (CFL step)
template <int EQ, int D>
__global__ void __launch_bounds__(NTHREADS) k_wave(Grid g, int l)
{
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

static int grid_for(const Grid& g, int l)
{
    long long b = (g.N[l] + NTHREADS - 1) / NTHREADS;
    return (int)(b < 1216 ? (b < 1 ? 1 : b) : 1216);
}

template <int EQ, int D>
static void stage_dispatch(const Grid& g, cudaStream_t st, int u, int s, int lmin, double dtl,
                           double bw, int reg)
{
    k_stage<EQ, D><<<grid_for(g, u), NTHREADS, 0, st>>>(g, u, s, lmin, dtl, bw, reg);
}

void launch_stage(const Grid& g, cudaStream_t st, int u, int s, int lmin, double dtl, double bw, int reg)
{
#define MRLT_CASE(E, DD) \
    if (g.eq == E && g.d == DD) return stage_dispatch<E, DD>(g, st, u, s, lmin, dtl, bw, reg);
    MRLT_CASE(0, 1) MRLT_CASE(0, 2) MRLT_CASE(0, 3)
    MRLT_CASE(1, 1) MRLT_CASE(1, 2) MRLT_CASE(1, 3)
    MRLT_CASE(2, 1) MRLT_CASE(2, 2) MRLT_CASE(2, 3)
    MRLT_CASE(3, 1) MRLT_CASE(3, 2) MRLT_CASE(3, 3)
#undef MRLT_CASE
}

void launch_wave(const Grid& g, cudaStream_t st, int l)
{
#define MRLT_CASE(E, DD) \
    if (g.eq == E && g.d == DD) {                                           \
        k_wave<E, DD><<<grid_for(g, l), NTHREADS, 0, st>>>(g, l);           \
        return;                                                             \
    }
    MRLT_CASE(0, 1) MRLT_CASE(0, 2) MRLT_CASE(0, 3)
    MRLT_CASE(1, 1) MRLT_CASE(1, 2) MRLT_CASE(1, 3)
    MRLT_CASE(2, 1) MRLT_CASE(2, 2) MRLT_CASE(2, 3)
    MRLT_CASE(3, 1) MRLT_CASE(3, 2) MRLT_CASE(3, 3)
#undef MRLT_CASE
}

} // namespace mrlt

// mrlt_api.cu -- host side of the C-ABI declared in include/mrlt.h: memory
// layout, the LT iteration schedule (Alg. 3), the global-step MR iteration,
// macro steps with the CFL rule, and read-back.
#include "mrlt.h"
#include "mrlt_macro.cuh"
#include "mrlt_tree.cuh"

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>
#include <chrono>
#include <mutex>
#include <thread>

using namespace mrlt;

struct mr_solver {
    mr_config cfg{};
    Launcher K;
    cudaStream_t stream = nullptr;
    std::vector<void*> allocs;      // fixed arrays (per cell, per level, scalars)
    std::vector<void*> node_allocs; // node arrays of the current capacity
    double* d_part = nullptr;
    long long ntot = 0;             // cells over all levels
    size_t fixed_bytes = 0;         // device bytes of the fixed arrays
    int* h_top = nullptr;           // pinned: [0] free slots, [1] refinement flags of a head,
                                    // [2..3] halt record (Grid::room[1..2])
    int* d_nref = nullptr;          // device: refinement flags counted by a head
    long long used_macro = 0;       // nodes of the tree installed at the macro step's start
    long long grow_macro = 0;       // largest growth past used_macro seen in this macro step
    // head of a macro step: iteration 0 up to the flags of its new tree (and
    // their count), run before the capacity check at the boundary
    bool head_pending = false;      // enqueued, its count not yet applied
    bool head_done = false;         // applied: iteration 0 continues with the tree's installation
    cudaGraphExec_t head_exec = nullptr;
    long long head_launches = 0;
    // a remesh that did not fit halted the device work (see halted()): the
    // host resumes at the halted iteration (resume: with the installation of
    // its tree) and launches `redo` iterations again without counting them
    bool resume = false;
    long long redo = 0;
    bool unchecked = false;         // iterations launched since the last check point
    long long halts = 0;            // halts recovered (statistics)
    long long reserved = 0;         // mr_reserve_nodes: capacity floor
    double t = 0.0, dt = 0.0;
    long long iters = 0, macros = 0, pos = 0, stage_launches = 0;
    bool reg = false;
    bool launch_failed = false; // a stage launch could not be configured
    std::string err;
    // stage-kernel timing (mr_profile)
    bool prof = false;
    std::vector<cudaEvent_t> ev;   // pairs: start 2i, stop 2i+1
    int ev_used = 0;
    std::vector<int> ev_level;     // level of each recorded pair
    double prof_ms = 0.0;
    double prof_level_ms[LMAX + 1] = {};
    long long prof_launches = 0, prof_all0 = 0;
    unsigned long long work0[(LMAX + 1) * 4] = {};
    // one macro step (2^{L-min} fine iterations) captured as a CUDA graph and
    // replayed on `stream`; captured on an internal stream because the legacy
    // default stream cannot be captured
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t macro_exec = nullptr;
    long long macro_launches = 0, macro_stage_launches = 0;
    bool graph_off = false; // capture failed once, or disabled by the caller
    // batched use: the macro-step finiteness check copies the device error
    // bits here (pinned host memory) instead of synchronising
    int* async_err = nullptr;
    // mr_set_async: calls return without waiting; own_err is the solver's own
    // pinned slot for async_err (batches and servers use theirs)
    bool async = false;
    int* own_err = nullptr;
    // device bytes requested by dev_alloc; with dry set nothing is allocated
    // (the footprint of a configuration is projected without creating it)
    size_t bytes = 0;
    bool dry = false;
    // launch mode: MR_LAUNCH_GRAPH (the default) launches one kernel per phase,
    // macro steps replayed as CUDA graphs; MR_LAUNCH_PERSISTENT runs the fine
    // iterations in one cooperative macro-step kernel (mrlt_macro.cuh)
    int launch_mode = MR_LAUNCH_GRAPH;
    unsigned* d_bar = nullptr;                 // grid barrier of the macro-step kernel
    bool wmax_valid = false;                   // g.wmax holds the CFL speed of the current state
    unsigned long long* d_stamps = nullptr;    // profiling stamps of the macro-step kernel
    int* d_nstamps = nullptr;
    double grid_wait_s = 4.0;                  // longest grid-barrier wait
};

namespace {

const char* kNullErr = "null handle";

#define MR_CK(call)                                                               \
    do {                                                                          \
        cudaError_t e_ = (call);                                                  \
        if (e_ != cudaSuccess) {                                                  \
            h->err = std::string(#call) + ": " + cudaGetErrorString(e_);          \
            return MR_E_CUDA;                                                     \
        }                                                                         \
    } while (0)

#define MR_TRY(expr)                 \
    do {                             \
        mr_status r_ = (expr);       \
        if (r_ != MR_OK) return r_;  \
    } while (0)

mr_status validate(const mr_config* c)
{
    if (!c) return MR_E_INVALID;
    if (c->dim < 1 || c->dim > 3) return MR_E_INVALID;
    if (c->max_level < 1 || c->max_level > LMAX || c->dim * c->max_level > 30) return MR_E_INVALID;
    if (c->min_level < 0 || c->min_level > c->max_level) return MR_E_INVALID;
    if (c->equation < 0 || c->equation > 3) return MR_E_INVALID;
    if (c->rk_order != 2 && c->rk_order != 3) return MR_E_INVALID;
    if (c->time_mode != MR_TIME_GTS && c->time_mode != MR_TIME_LT_NERK) return MR_E_INVALID;
    if (c->precision != MR_PREC_FP64 && c->precision != MR_PREC_MIXED) return MR_E_INVALID;
    if (c->flux != MR_FLUX_DEFAULT && !(c->flux == MR_FLUX_AUSM_PLUS && c->equation == MR_EQ_EULER))
        return MR_E_INVALID;
    if (c->adapt_mode < 0 || c->adapt_mode > 2) return MR_E_INVALID;
    if (!(c->cfl > 0.0) || !(c->eps >= 0.0)) return MR_E_INVALID;
    for (int k = 0; k < c->dim; ++k) {
        if (!(c->hi[k] > c->lo[k])) return MR_E_INVALID;
        if (c->bc[k] != MR_BC_PERIODIC && c->bc[k] != MR_BC_NEUMANN && c->bc[k] != MR_BC_DIRICHLET0)
            return MR_E_INVALID;
        if (c->bc[k] == MR_BC_DIRICHLET0 && c->equation == MR_EQ_EULER) return MR_E_INVALID;
    }
    if (c->equation == MR_EQ_EULER && !(c->phys[0] > 1.0)) return MR_E_INVALID;
    return MR_OK;
}

// Solver memory comes from a library-private, stream-ordered memory pool per
// device that keeps freed memory cached: creating and destroying solvers
// (batches, a server admitting and releasing requests) then never calls
// cudaMalloc or cudaFree, whose device-wide synchronisation would stall the
// other solvers' work in flight.  The cached memory stays reserved until the
// process exits.
constexpr int kMaxPoolDevices = 64;
cudaMemPool_t g_pool[kMaxPoolDevices] = {};
std::mutex g_pool_mutex; // pools are created once per device, also under concurrent first use

cudaMemPool_t device_pool()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxPoolDevices) return nullptr;
    std::lock_guard<std::mutex> lock(g_pool_mutex);
    if (!g_pool[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        unsigned long long keep = ~0ull; // never release cached memory at synchronisation
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        g_pool[dev] = pool;
    }
    return g_pool[dev];
}

// bytes the pool holds cached (reserved, not in use) on the current device
size_t pool_cached_bytes()
{
    cudaMemPool_t pool = device_pool();
    unsigned long long reserved = 0, used = 0;
    if (!pool || cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved) != cudaSuccess ||
        cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return reserved > used ? (size_t)(reserved - used) : 0;
}

template <class T>
mr_status dev_alloc(mr_solver* h, T** p, size_t count)
{
    *p = nullptr;
    if (count == 0) return MR_OK;
    h->bytes += (count * sizeof(T) + 255) / 256 * 256;
    if (h->dry) return MR_OK;
    cudaMemPool_t pool = device_pool();
    cudaError_t e = pool ? cudaMallocFromPoolAsync((void**)p, count * sizeof(T), pool, h->stream)
                         : cudaErrorMemoryAllocation;
    if (e != cudaSuccess) {
        h->err = std::string("device allocation: ") + cudaGetErrorString(e);
        *p = nullptr;
        cudaGetLastError();
        return MR_E_NOMEM;
    }
    h->allocs.push_back(*p);
    return MR_OK;
}

// ---------------------------------------------------------------- node storage
// Node values live in arrays of `cap` slots (see mrlt_impl.cuh).  A new tree
// (creation, reset, a full adaptation, an installed tree) gets room for every
// cell of every level.  A solver whose full arrays cost at most kDenseBytes
// keeps them, and so does the persistent launch mode; any other is resized
// at macro-step boundaries, where the size of the next tree is known
// exactly: the first fine iteration of a macro step, which holds its only
// full remesh, is split after the adaptation has flagged the new tree (the
// head of the macro step).  The flags are counted (every refined cell owns
// 2^d children), the count is read back together with the CFL speed, and
// the arrays are resized before the tree is installed.  With need = max(nodes
// in use, nodes of the next tree) and margin = max(2 x the largest growth seen
// within the last macro step, a quarter of need, kMinSlots), arrays with
// fewer than need + margin or more than need + 4 margin slots are set to
// need + 2 margin.  Inside a macro step (adaptation at every fine iteration,
// on the levels that are active) every remesh first checks on the device
// that its tree fits, and halts the solver's device work if it does not
// (room_decide).  The host reads the halt record at the end of the macro step (a
// solver that waits) or with the CFL speed at the next boundary (batch and
// server instances); after a halt it grows the arrays to the flagged tree
// plus two margins of max(a quarter of it, 2 x its growth since the macro
// step began) and resumes at the halted remesh.
// Reservations made with mr_reserve_nodes are a floor.
constexpr long long kMinSlots = 4096;
constexpr size_t kDenseBytes = 32u << 20;

size_t per_node_bytes(const Grid& g, bool reg)
{
    const size_t esz = g.prec ? sizeof(float) : sizeof(double);
    return NFIELD * g.m * esz + (reg ? (size_t)g.nf * g.m * sizeof(double) : 0) + sizeof(int);
}

// new node arrays of cap slots into g (fields, registers, free stack);
// the previous pointers are not freed here
mr_status alloc_nodes(mr_solver* h, Grid& g, long long cap, std::vector<void*>& out)
{
    cudaMemPool_t pool = device_pool();
    auto take = [&](void** p, size_t bytes) -> bool {
        *p = nullptr;
        if (!pool || cudaMallocFromPoolAsync(p, bytes, pool, h->stream) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        out.push_back(*p);
        return true;
    };
    const size_t esz = g.prec ? sizeof(float) : sizeof(double);
    bool ok = true;
    for (int f = 0; f < NFIELD && ok; ++f) ok = take(&g.f[f], (size_t)cap * g.m * esz);
    if (ok && h->reg) {
        ok = take((void**)&g.rg, (size_t)cap * g.nf * g.m * sizeof(double));
    } else if (ok) {
        g.rg = nullptr;
    }
    if (ok) ok = take((void**)&g.fstack, (size_t)cap * sizeof(int));
    if (!ok) {
        h->err = "device allocation of node arrays failed";
        return MR_E_NOMEM;
    }
    g.cap = cap;
    return MR_OK;
}

void drop_graphs(mr_solver* h);

void free_allocs(mr_solver* h, std::vector<void*>& v)
{
    for (void* p : v) cudaFreeAsync(p, h->stream);
    v.clear();
}

// Replace the node arrays by arrays of newcap slots.  keep: copy the live
// nodes (compacted into slots 1..used, in level and list order); otherwise
// the arrays are fresh (the caller initialises them).  A captured macro step
// holds the old pointers, so it is dropped.
mr_status set_capacity(mr_solver* h, long long newcap, bool keep)
{
    Grid& g = h->K.g;
    if (newcap > h->ntot + 1) newcap = h->ntot + 1;
    if (newcap == g.cap) return MR_OK;
    int cnt[2 * (LMAX + 1)] = {};
    long long used = 0;
    if (keep) {
        MR_CK(cudaMemcpyAsync(cnt, g.counts, sizeof cnt, cudaMemcpyDeviceToHost, h->stream));
        MR_CK(cudaStreamSynchronize(h->stream));
        for (int l = g.lb; l <= g.L; ++l) used += cnt[l] + cnt[LMAX + 1 + l];
        if (used + 1 > newcap) newcap = used + 1;
    }
    if (h->macro_exec || h->head_exec) { // captured with the old arrays
        MR_CK(cudaStreamSynchronize(h->stream));
        drop_graphs(h);
    }
    const Grid from = g;
    Grid ng = g; // the solver keeps its arrays if an allocation fails
    std::vector<void*> fresh;
    const mr_status ra = alloc_nodes(h, ng, newcap, fresh);
    if (ra != MR_OK) {
        free_allocs(h, fresh);
        return ra;
    }
    g = ng;
    if (keep) h->K.renumber(from, cnt, used);
    free_allocs(h, h->node_allocs);
    h->node_allocs.swap(fresh);
    h->bytes = h->fixed_bytes + (size_t)newcap * per_node_bytes(g, h->reg);
    MR_CK(cudaGetLastError());
    return MR_OK;
}

// node arrays with a slot for every cell (no resizing needed)
bool dense_capacity(const mr_solver* h) { return h->K.g.cap >= h->ntot + 1; }

// room for every cell is cheap enough to keep
bool small_problem(const mr_solver* h)
{
    return (size_t)(h->ntot + 1) * per_node_bytes(h->K.g, h->reg) <= kDenseBytes;
}

// the macro step's head is split off iteration 0 (see the capacity rule)
bool split_head(const mr_solver* h)
{
    return h->cfg.adapt_mode != MR_ADAPT_NEVER && !small_problem(h) && h->launch_mode == MR_LAUNCH_GRAPH;
}

// remeshes inside macro steps check that their trees fit (and halt if not)
bool can_halt(const mr_solver* h)
{
    return split_head(h) && h->cfg.adapt_mode == MR_ADAPT_EVERY;
}

// The capacity rule at a macro-step boundary, with the free-slot count `top`
// read back; next = nodes of the tree its head flagged, or -1 when the tree
// does not change there.
mr_status adjust_capacity(mr_solver* h, int top, long long next = -1)
{
    if ((small_problem(h) || h->launch_mode == MR_LAUNCH_PERSISTENT) && dense_capacity(h)) return MR_OK;
    const long long cap = h->K.g.cap, used = cap - 1 - top;
    auto clamp = [&](long long t) {
        if (t < h->reserved + 1) t = h->reserved + 1;
        return t > h->ntot + 1 ? h->ntot + 1 : t;
    };
    auto at_least = [](long long a, long long b) { return a > b ? a : b; };
    if (used - h->used_macro > h->grow_macro) h->grow_macro = used - h->used_macro;
    const long long need = at_least(used, next);
    const long long margin = at_least(at_least(2 * h->grow_macro, need / 4), kMinSlots);
    const long long target = clamp(need + 2 * margin + 1);
    h->used_macro = next >= 0 ? next : used;
    h->grow_macro = 0;
    if (cap - 1 < need + margin || cap - 1 > need + 4 * margin) return set_capacity(h, target, true);
    return MR_OK;
}

// nodes in use (a synchronising read of the lists' counts)
mr_status count_nodes(mr_solver* h, long long* used)
{
    int cnt[2 * (LMAX + 1)] = {};
    MR_CK(cudaMemcpyAsync(cnt, h->K.g.counts, sizeof cnt, cudaMemcpyDeviceToHost, h->stream));
    MR_CK(cudaStreamSynchronize(h->stream));
    *used = 0;
    for (int l = h->K.g.lb; l <= h->K.g.L; ++l) *used += cnt[l] + cnt[LMAX + 1 + l];
    return MR_OK;
}

// end of a call that built a new tree (held in arrays with room for every
// cell until the next macro-step boundary)
mr_status fit_new_tree(mr_solver* h)
{
    MR_CK(cudaMemsetAsync(h->K.g.flag, 0, (size_t)h->ntot, h->stream)); // (see adapt)
    long long used = 0;
    MR_TRY(count_nodes(h, &used));
    h->used_macro = used;
    h->grow_macro = 0;
    h->head_pending = h->head_done = false;
    return MR_OK;
}

// a batch or server instance: its progress is driven by events, not waits
bool is_instance(const mr_solver* h) { return h->async_err && h->async_err != h->own_err; }

// Recovery from a halt whose record (h_top[2..3]) and free-slot count
// (h_top[0]) were read back with the stream idle: the halt at iteration p
// is cleared, the arrays grow to hold the flagged tree and two margins (see
// the capacity rule), and the position rewinds to p (into the macro step just
// counted complete, when pos is 0).  The caller then resumes with the
// installation of p's tree (its flags are intact: nothing ran after them)
// and launches the iterations after p again (h->redo, not counted twice).
mr_status recover(mr_solver* h)
{
    Grid& g = h->K.g;
    const long long nit = 1LL << (g.L - g.lb);
    const long long p = h->h_top[2] - 1, tree = h->h_top[3];
    const long long launched = h->pos == 0 ? nit : h->pos;
    if (p < 1 || p >= launched) {
        h->err = "halt record out of range";
        return MR_E_STATE;
    }
    const long long used = g.cap - 1 - h->h_top[0];
    const long long need = tree > used ? tree : used;
    long long margin = need / 4;
    if (margin < 2 * (need - h->used_macro)) margin = 2 * (need - h->used_macro); // a fast-growing tree
    if (margin < kMinSlots) margin = kMinSlots;
    long long target = need + 2 * margin + 1;
    if (target < h->reserved + 1) target = h->reserved + 1;
    // grown first: if that fails the solver stays halted, and a later call retries
    MR_TRY(set_capacity(h, target, true));
    MR_CK(cudaMemsetAsync(g.room, 0, 4 * sizeof(int), h->stream));
    h->h_top[2] = h->h_top[3] = 0;
    if (h->pos == 0) {
        --h->macros;
        h->head_pending = h->head_done = false; // the boundary's head ran halted: again
    }
    if (need - h->used_macro > h->grow_macro) h->grow_macro = need - h->used_macro;
    h->redo += launched - p;
    h->pos = p;
    h->resume = true;
    ++h->halts;
    return MR_OK;
}

// the free-slot count and the halt record on their way to h_top
mr_status enqueue_slot_record(mr_solver* h)
{
    MR_CK(cudaMemcpyAsync(h->h_top, h->K.g.ftop, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    MR_CK(cudaMemcpyAsync(h->h_top + 2, h->K.g.room + 1, 2 * sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    return MR_OK;
}

// A check point at the end of a macro step or call (synchronising): after
// a halt the position rewinds (*rewound).
mr_status check_point(mr_solver* h, bool* rewound)
{
    *rewound = false;
    MR_TRY(enqueue_slot_record(h));
    MR_CK(cudaStreamSynchronize(h->stream));
    if (!h->h_top[2]) return MR_OK;
    MR_TRY(recover(h));
    *rewound = true;
    return MR_OK;
}

mr_status run_iters(mr_solver* h, double dt, long long n);

void drop_graphs(mr_solver* h)
{
    if (h->macro_exec) cudaGraphExecDestroy(h->macro_exec);
    h->macro_exec = nullptr;
    if (h->head_exec) cudaGraphExecDestroy(h->head_exec);
    h->head_exec = nullptr;
}

// transient device scratch from the pool, released in stream order
template <class T>
mr_status scratch(mr_solver* h, T** p, size_t count)
{
    *p = nullptr;
    cudaMemPool_t pool = device_pool();
    if (!pool || cudaMallocFromPoolAsync((void**)p, count * sizeof(T) + 16, pool, h->stream) != cudaSuccess) {
        cudaGetLastError();
        h->err = "device allocation of scratch memory failed";
        return MR_E_NOMEM;
    }
    return MR_OK;
}

int level_min(const mr_solver* h, long long n)
{
    const Grid& g = h->K.g;
    for (int l = g.lb; l <= g.L; ++l)
        if (n % (1LL << (g.L - l)) == 0) return l;
    return g.L;
}

// add the elapsed times of the recorded event pairs to the running total
void drain_events(mr_solver* h)
{
    if (h->ev_used == 0) return;
    cudaEventSynchronize(h->ev[2 * h->ev_used - 1]);
    for (int i = 0; i < h->ev_used; ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, h->ev[2 * i], h->ev[2 * i + 1]) == cudaSuccess) {
            h->prof_ms += ms;
            h->prof_level_ms[h->ev_level[i]] += ms;
        }
    }
    h->ev_used = 0;
}

// one compact RK stage s on the leaves of levels lo..hi (one launch when the
// levels are independent); dt is the finest-level step
void stage(mr_solver* h, int lo, int hi, int s, int lmin)
{
    const Grid& g = h->K.g;
    static const double b2[2] = {0.5, 0.5};
    static const double b3[3] = {1.0 / 6.0, 1.0 / 6.0, 2.0 / 3.0};
    const double b = g.rk == 2 ? b2[s - 1] : b3[s - 1];
    const int reg = h->reg && !g.gts;
    int launched;
    if (h->prof) {
        if (h->ev_used * 2 + 2 > (int)h->ev.size()) drain_events(h);
        cudaEventRecord(h->ev[2 * h->ev_used], h->stream);
        h->ev_level[h->ev_used] = hi;
        launched = launch_stage(g, h->stream, lo, hi, s, lmin, b, reg);
        cudaEventRecord(h->ev[2 * h->ev_used + 1], h->stream);
        ++h->ev_used;
        h->prof_launches += launched > 0 ? launched : 0;
    } else {
        launched = launch_stage(g, h->stream, lo, hi, s, lmin, b, reg);
    }
    if (launched < 0) {
        h->launch_failed = true;
        return;
    }
    h->stage_launches += launched;
}

mr_status sync_check(mr_solver* h)
{
    if (h->launch_failed) {
        h->launch_failed = false;
        h->err = "stage kernel could not be configured (shared memory or occupancy query failed)";
        return MR_E_CUDA;
    }
    MR_CK(cudaGetLastError());
    int e = 0;
    MR_CK(cudaMemcpyAsync(&e, h->K.g.err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    MR_CK(cudaStreamSynchronize(h->stream));
    if (e) {
        char buf[128];
        snprintf(buf, sizeof buf, "device reported error bits 0x%x%s", e,
                 (e & ERR_TIMEOUT) ? " (a grid barrier wait gave up)" : "");
        h->err = buf;
        if (e & ERR_TIMEOUT) return MR_E_TIMEOUT;
        if (e & ERR_CAPACITY) {
            h->err += " (node capacity exhausted within a macro step: the tree more than doubled; "
                      "reserve more nodes with mr_reserve_nodes)";
            return MR_E_NOMEM;
        }
        return (e & ERR_NONFINITE) ? MR_E_NUMERIC : MR_E_STATE;
    }
    return MR_OK;
}

// Algs. 1-2 restricted to levels >= la (full adaptation for la = min_level)
// part 1: details, thresholds and closure (the new tree in the flags); part
// 2: the tree installed (slots released and taken), lists, projections; 0:
// both.  A caller may check the node capacity between the parts.
mr_status adapt(mr_solver* h, int la, int part = 0, long long it = 0)
{
    Grid& g = h->K.g;
    if (la >= g.L) return MR_OK;
    if (part != 2) {
        if (la == g.lb) {
            h->K.scale_init();
            for (int l = g.lb; l <= g.L; ++l) h->K.scale(l);
        }
        // the flags are zero here: every remesh's compaction clears those it set
        h->K.mark_refinements(la, part == 0 && can_halt(h) ? it : -1);
    }
    if (part != 1) {
        h->K.apply_tree(la);
        h->K.compact(la, g.L);
        h->K.project_up(g.L - 1, la, PM_Q0);
    }
    return MR_OK;
}

// one iteration n (0-based in the macro step) of Alg. 3
// part 1 ends inside the adaptation, before the new tree is installed;
// part 2 continues from there (see adapt); 0: the whole iteration
mr_status lt_iteration(mr_solver* h, long long n, long long nit, int part = 0)
{
    Grid& g = h->K.g;
    const int L = g.L, lb = g.lb, lmin = level_min(h, n);
    if (part != 2) {
        h->K.leaf_copy(lmin, L, F_QE, F_Q0);
        h->K.project_up(L - 1, lmin, PM_Q0);
    }
    if (h->cfg.adapt_mode == MR_ADAPT_EVERY || (h->cfg.adapt_mode == MR_ADAPT_MACRO && n == 0))
        MR_TRY(adapt(h, lmin, part, n));
    if (part == 1) return MR_OK;
    if (lmin > lb) h->K.project(lmin - 1, PM_MID);
    stage(h, lmin, L, 1, lmin); // first stage: all active levels at once
    h->K.project_up(L - 1, lmin, PM_REF2);
    for (int l = L; l >= lmin; --l) {
        if (l < L) h->K.project(l, PM_PRJ2);
        stage(h, l, l, 2, lmin);
    }
    if (g.rk == 3) {
        h->K.project_up(L - 1, lmin, PM_REF3);
        for (int l = L; l >= lmin; --l) {
            if (l < L) h->K.project(l, PM_PRJ3);
            stage(h, l, l, 3, lmin);
        }
    }
    if (h->reg) {
        const int lc = (n + 1 == nit) ? lb : level_min(h, n + 1);
        if (lc < L) h->K.reflux(lc, L - 1);
    }
    return MR_OK;
}

// global time step MR (MR/RK2, MR/RK3)
mr_status gts_iteration(mr_solver* h, long long n, int part = 0)
{
    Grid& g = h->K.g;
    const int L = g.L, lb = g.lb;
    if (part != 2) {
        h->K.leaf_copy(lb, L, F_QE, F_Q0);
        h->K.project_up(L - 1, lb, PM_Q0);
    }
    if (h->cfg.adapt_mode == MR_ADAPT_EVERY || (h->cfg.adapt_mode == MR_ADAPT_MACRO && n == 0))
        MR_TRY(adapt(h, lb, part, n));
    if (part == 1) return MR_OK;
    stage(h, lb, L, 1, lb); // every level at the same instant: one launch per stage
    h->K.project_up(L - 1, lb, PM_Q1);
    stage(h, lb, L, 2, lb);
    if (g.rk == 3) {
        h->K.project_up(L - 1, lb, PM_Q2);
        stage(h, lb, L, 3, lb);
    }
    return MR_OK;
}

mr_status finite_check(mr_solver* h)
{
    for (int l = h->K.g.lb; l <= h->K.g.L; ++l) h->K.finite(l);
    if (h->async_err) {
        MR_CK(cudaMemcpyAsync(h->async_err, h->K.g.err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        return MR_OK;
    }
    return sync_check(h);
}

mr_status iteration(mr_solver* h, long long n, long long nit, int part = 0)
{
    return h->K.g.gts ? gts_iteration(h, n, part) : lt_iteration(h, n, nit, part);
}

// the part of iteration n that a macro step runs after its head (see the
// capacity rule): the rest of iteration 0 when the head was split off
int part_of(const mr_solver* h, long long n) { return n == 0 && split_head(h) ? 2 : 0; }

// Capture what `body` enqueues as a CUDA graph (stream capture on the
// internal stream).  Every launch of a macro step is fixed by the layout,
// the level schedule l_min(n) and the configuration; the fine step is read
// from g.dtp, so one graph serves every macro step.  Returns false (and
// leaves nothing captured) when capture is not possible; the caller then
// launches directly.
template <class Body>
bool capture(mr_solver* h, Body body, cudaGraphExec_t* exec, long long* launches, long long* stage_launches)
{
    if (!h->cap_stream && cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    // stage-kernel attributes and occupancy are set up before capture begins
    if (launch_stage(h->K.g, h->stream, 1, 0, 1, 0, 0.0, 0) < 0) return false;
    cudaStream_t user = h->stream;
    const long long k0 = h->K.n, s0 = h->stage_launches;
    h->stream = h->K.st = h->cap_stream;
    bool ok = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    const mr_status r = ok ? body() : MR_OK;
    cudaGraph_t graph = nullptr;
    if (ok) ok = cudaStreamEndCapture(h->cap_stream, &graph) == cudaSuccess && r == MR_OK && !h->launch_failed;
    h->stream = h->K.st = user;
    h->launch_failed = false;
    *exec = nullptr;
    if (ok) ok = cudaGraphInstantiate(exec, graph, 0) == cudaSuccess;
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError(); // clear a capture error so that the direct path starts clean
    *launches = h->K.n - k0;
    if (stage_launches) *stage_launches = h->stage_launches - s0;
    h->K.n = k0;
    h->stage_launches = s0;
    if (!ok) *exec = nullptr;
    return ok;
}

// fine iterations [n0, n0 + cnt) of a macro step (iteration 0 from its head on)
bool capture_iters(mr_solver* h, long long n0, long long cnt, long long nit, cudaGraphExec_t* exec,
                   long long* launches, long long* stage_launches)
{
    auto body = [&]() -> mr_status {
        for (long long i = n0; i < n0 + cnt; ++i) MR_TRY(iteration(h, i, nit, part_of(h, i)));
        return MR_OK;
    };
    return capture(h, body, exec, launches, stage_launches);
}

bool capture_macro(mr_solver* h, long long nit)
{
    return capture_iters(h, 0, nit, nit, &h->macro_exec, &h->macro_launches, &h->macro_stage_launches);
}

// The head of the next macro step (iteration 0 up to the flags of the new
// tree, and their count) enqueued, the count and the free-slot count on
// their way to h_top; head_finish applies them once the stream has passed.
mr_status head_enqueue(mr_solver* h)
{
    if (!split_head(h) || h->head_done || h->head_pending) return MR_OK;
    const long long nit = 1LL << (h->K.g.L - h->K.g.lb);
    auto body = [&]() -> mr_status {
        MR_TRY(iteration(h, 0, nit, 1));
        h->K.count_refined(h->K.g.lb, h->d_nref);
        return MR_OK;
    };
    bool graphed = false;
    if (!h->prof && !h->graph_off) {
        if (h->head_exec || capture(h, body, &h->head_exec, &h->head_launches, nullptr)) {
            MR_CK(cudaGraphLaunch(h->head_exec, h->stream));
            h->K.n += h->head_launches;
            graphed = true;
        } else {
            h->graph_off = true;
        }
    }
    if (!graphed) MR_TRY(body());
    MR_CK(cudaMemcpyAsync(h->h_top + 1, h->d_nref, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    MR_CK(cudaMemcpyAsync(h->h_top, h->K.g.ftop, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    h->head_pending = true;
    return MR_OK;
}

// the capacity rule at a macro-step boundary, once h_top holds what the
// head (if any) and the free-slot read enqueued before it
mr_status head_finish(mr_solver* h)
{
    if (!h->head_pending) return adjust_capacity(h, h->h_top[0]);
    h->head_pending = false;
    h->head_done = true;
    const Grid& g = h->K.g;
    const long long next = g.N[g.lb] + ((long long)h->h_top[1] << g.d);
    return adjust_capacity(h, h->h_top[0], next);
}

// head and capacity rule of a macro-step boundary, synchronously
mr_status boundary_check(mr_solver* h)
{
    MR_TRY(head_enqueue(h));
    MR_TRY(enqueue_slot_record(h));
    MR_TRY(sync_check(h));
    if (h->h_top[2]) { // check points end every macro step of a solver that waits
        h->err = "halt pending at a macro-step boundary";
        return MR_E_STATE;
    }
    return head_finish(h);
}

// Graphs are used for whole macro steps with profiling off, up to 1024 fine
// iterations per macro step (larger schedules launch directly).
constexpr long long kMaxGraphIters = 1024;

// Profiling capacity of the macro-step kernel's phase stamps; a profiled run
// launches at most kProfIters fine iterations per macro-step kernel.
constexpr int kStampCap = 1 << 15;
constexpr long long kProfIters = 256;

// Sum the stage phases recorded by the last profiled macro-step kernel:
// the duration of a phase is the time from its start to the next phase's.
mr_status drain_stamps(mr_solver* h)
{
    int n = 0;
    MR_CK(cudaMemcpyAsync(&n, h->d_nstamps, sizeof n, cudaMemcpyDeviceToHost, h->stream));
    MR_CK(cudaStreamSynchronize(h->stream));
    if (n > kStampCap) n = kStampCap;
    std::vector<unsigned long long> st((size_t)2 * n);
    if (n) MR_CK(cudaMemcpyAsync(st.data(), h->d_stamps, st.size() * sizeof(unsigned long long),
                                 cudaMemcpyDeviceToHost, h->stream));
    MR_CK(cudaStreamSynchronize(h->stream));
    for (int i = 0; i + 1 < n; ++i) {
        const int kind = (int)(st[2 * i] >> 8), level = (int)(st[2 * i] & 255);
        if (kind < PH_STAGE1 || kind > PH_STAGE3) continue;
        const double ms = (double)(st[2 * i + 3] - st[2 * i + 1]) * 1e-6;
        h->prof_ms += ms;
        if (level <= LMAX) h->prof_level_ms[level] += ms;
        ++h->prof_launches;
    }
    return MR_OK;
}

// Iterations [pos, pos + count) of the current macro step in one launch of
// the persistent macro-step kernel (count <= nit - pos).
mr_status run_persistent(mr_solver* h, long long count, long long nit)
{
    MacroArgs a = {};
    a.n0 = h->pos;
    a.n1 = h->pos + count;
    a.nit = nit;
    a.adapt_mode = h->cfg.adapt_mode;
    a.reg = h->reg && !h->K.g.gts;
    a.end_of_macro = a.n1 == nit;
    a.bar = h->d_bar;
    a.limit_ns = (unsigned long long)(h->grid_wait_s * 1e9);
    a.bc = h->K.bc;
    if (h->prof) {
        a.stamps = h->d_stamps;
        a.nstamps = h->d_nstamps;
        a.stamp_cap = kStampCap;
        MR_CK(cudaMemsetAsync(h->d_nstamps, 0, sizeof(int), h->stream));
    }
    MR_CK(cudaMemsetAsync(h->d_bar, 0, 2 * sizeof(unsigned), h->stream));
    if (launch_macro(h->K.g, h->stream, &a) < 0) {
        cudaGetLastError();
        h->err = "macro-step kernel could not be launched (cooperative launch or occupancy query failed)";
        return MR_E_CUDA;
    }
    ++h->K.n;
    h->wmax_valid = false;
    if (h->prof) MR_TRY(drain_stamps(h));
    return MR_OK;
}

mr_status run_iters(mr_solver* h, double dt, long long n)
{
    const long long nit = 1LL << (h->K.g.L - h->K.g.lb);
    if (h->pos != 0 && dt != h->dt) {
        h->err = "dt changed inside a macro step";
        return MR_E_STATE;
    }
    h->dt = dt;
    long long i = 0; // new iterations launched by this call
    // k iterations launched from h->pos (the first ones again after a halt)
    auto advance = [&](long long k) {
        const long long fresh = k > h->redo ? k - h->redo : 0;
        h->redo = h->redo > k ? h->redo - k : 0;
        h->iters += fresh;
        i += fresh;
        h->pos += k;
        h->head_done = h->resume = false;
        // batch and server instances learn of a halt at their next boundary
        h->unchecked = can_halt(h) && !dense_capacity(h) && !is_instance(h);
    };
    for (;;) {
        const bool done = i >= n && h->redo == 0;
        // check points: the end of a macro step and the end of this call
        // (compact arrays, remeshes at every fine iteration)
        if (h->unchecked && (h->pos == nit || done)) {
            h->unchecked = false;
            bool rewound = false;
            MR_TRY(check_point(h, &rewound));
            if (rewound) continue;
        }
        if (h->pos == nit) { // every iteration of the macro step launched
            h->pos = 0;
            ++h->macros;
            if (h->launch_mode != MR_LAUNCH_PERSISTENT) {
                MR_TRY(finite_check(h));
            } else {
                h->wmax_valid = true; // the kernel ended with the CFL reduction
                if (h->async_err) {
                    MR_CK(cudaMemcpyAsync(h->async_err, h->K.g.err, sizeof(int), cudaMemcpyDeviceToHost,
                                          h->stream));
                } else {
                    MR_TRY(sync_check(h));
                }
            }
        }
        if (i >= n && h->redo == 0) break;
        if (h->pos == 0) {
            if (split_head(h) && !h->head_done) MR_TRY(boundary_check(h));
            h->K.set_dt(dt);
        }
        if (h->resume) { // the halted iteration from its tree's installation on
            MR_TRY(iteration(h, h->pos, nit, 2));
            h->wmax_valid = false;
            advance(1);
            continue;
        }
        const long long left = n - i + h->redo; // iterations still to launch
        if (h->launch_mode == MR_LAUNCH_PERSISTENT) {
            long long chunk = left < nit - h->pos ? left : nit - h->pos;
            if (h->prof && chunk > kProfIters) chunk = kProfIters;
            MR_TRY(run_persistent(h, chunk, nit));
            advance(chunk);
            continue;
        }
        h->wmax_valid = false;
        const bool can_graph = !h->prof && !h->graph_off && nit <= kMaxGraphIters;
        if (can_graph && h->pos == 0 && left >= nit) { // a whole macro step
            if (!h->macro_exec && !capture_macro(h, nit)) {
                h->graph_off = true; // launch directly from now on
                continue;
            }
            MR_CK(cudaGraphLaunch(h->macro_exec, h->stream));
            h->K.n += h->macro_launches;
            h->stage_launches += h->macro_stage_launches;
            advance(nit);
            continue;
        }
        MR_TRY(iteration(h, h->pos, nit, part_of(h, h->pos)));
        advance(1);
    }
    return MR_OK;
}

// CFL step of the finest level: sigma * min(dx_L / max sum_k lambda_k, dx_L^2 / (2 d D))
// (the paper fixes only sigma; the step is held for a whole macro step)
// CFL reduction, enqueued: the largest sum of characteristic speeds,
// as a bit pattern, lands in *bits when the stream reaches this point
mr_status cfl_enqueue(mr_solver* h, unsigned long long* bits)
{
    Grid& g = h->K.g;
    // free node slots and the halt record, for the capacity rule at this boundary
    MR_TRY(enqueue_slot_record(h));
    if (h->wmax_valid) { // computed at the end of the macro-step kernel that led to this state
        MR_CK(cudaMemcpyAsync(bits, g.wmax, sizeof *bits, cudaMemcpyDeviceToHost, h->stream));
        return MR_OK;
    }
    MR_CK(cudaMemsetAsync(g.wmax, 0, sizeof(unsigned long long), h->stream));
    for (int l = g.lb; l <= g.L; ++l) {
        launch_wave(g, h->stream, l);
        ++h->stage_launches;
    }
    MR_CK(cudaMemcpyAsync(bits, g.wmax, sizeof *bits, cudaMemcpyDeviceToHost, h->stream));
    return MR_OK;
}

// fine step from the largest speed: cfl * dx_L / lambda, and for reaction-
// diffusion at most the explicit diffusion limit dx^2 / (2 d D)
double cfl_from_bits(const mr_solver* h, unsigned long long bits)
{
    const Grid& g = h->K.g;
    double lam;
    memcpy(&lam, &bits, sizeof lam);
    double dxm = g.dx[g.L][0];
    for (int k = 1; k < g.d; ++k) dxm = fmin(dxm, g.dx[g.L][k]);
    double d = lam > 0.0 ? dxm / lam : dxm;
    if (g.eq == MR_EQ_REACTION_DIFFUSION) {
        const double dd = dxm * dxm / (2.0 * g.d * g.phys[0]);
        if (lam <= 0.0 || dd < d) d = dd;
    }
    return h->cfg.cfl * d;
}

mr_status cfl_dt(mr_solver* h, double* dt)
{
    unsigned long long bits = 0;
    MR_TRY(cfl_enqueue(h, &bits));
    MR_TRY(sync_check(h));
    *dt = cfl_from_bits(h, bits);
    return MR_OK;
}

mr_status init_state(mr_solver* h, const double* q0)
{
    Grid& g = h->K.g;
    const int m = g.m;
    // the full tree: every cell of every level a node, then adapted
    MR_TRY(set_capacity(h, h->ntot + 1, false));
    const size_t esz = g.prec ? sizeof(float) : sizeof(double); // field element
    for (int f = 0; f < NFIELD; ++f) MR_CK(cudaMemsetAsync(g.f[f], 0, (size_t)g.cap * m * esz, h->stream));
    if (g.rg) MR_CK(cudaMemsetAsync(g.rg, 0, (size_t)g.cap * g.nf * m * sizeof(double), h->stream));
    MR_CK(cudaMemsetAsync(g.flag, 0, h->ntot, h->stream));
    MR_CK(cudaMemsetAsync(g.counts, 0, 3 * (LMAX + 1) * sizeof(int), h->stream));
    MR_CK(cudaMemsetAsync(g.err, 0, sizeof(int), h->stream));
    MR_CK(cudaMemsetAsync(g.room, 0, 4 * sizeof(int), h->stream));
    MR_CK(cudaMemsetAsync(g.near, 0, sizeof(unsigned long long), h->stream));
    MR_CK(cudaMemsetAsync(g.updates, 0, sizeof(unsigned long long), h->stream));
    for (int l = g.lb; l <= g.L; ++l)
        MR_CK(cudaMemsetAsync(g.st + g.off[l], l < g.L ? 2 : 1, (size_t)g.N[l], h->stream));
    h->K.slots_full(h->ntot);
    double* d_q = nullptr; // finest data through a transient double buffer, stored in the fields' type
    MR_TRY(scratch(h, &d_q, (size_t)g.N[g.L] * m));
    MR_CK(cudaMemcpyAsync(d_q, q0, (size_t)g.N[g.L] * m * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    h->K.store_finest(d_q);
    MR_CK(cudaFreeAsync(d_q, h->stream));
    h->K.compact(g.lb, g.L);
    for (int l = g.L - 1; l >= g.lb; --l) h->K.project(l, PM_Q0);
    if (h->cfg.adapt_mode != MR_ADAPT_NEVER) MR_TRY(adapt(h, g.lb));
    h->K.leaf_copy(g.lb, g.L, F_Q0, F_QE);
    h->t = h->dt = 0.0;
    h->iters = h->macros = h->pos = 0;
    h->wmax_valid = false;
    MR_TRY(sync_check(h));
    return fit_new_tree(h);
}

} // namespace

extern "C" {

} // extern "C"

namespace {

// Grid layout of a configuration and the device allocations of a solver
// (counted only, when h->dry is set).
mr_status layout_alloc(mr_solver* h, const mr_config* cfg)
{
    Grid& g = h->K.g;
    memset(&g, 0, sizeof g);
    g.d = cfg->dim;
    g.m = cfg->equation == MR_EQ_EULER ? cfg->dim + 2 : 1;
    g.nf = 2 * g.d;
    g.L = cfg->max_level;
    g.lb = cfg->min_level;
    g.eq = cfg->equation;
    g.rk = cfg->rk_order;
    g.gts = cfg->time_mode == MR_TIME_GTS;
    for (int k = 0; k < 3; ++k) g.bc[k] = cfg->bc[k];
    for (int k = 0; k < 8; ++k) g.phys[k] = cfg->phys[k];
    g.eps = cfg->eps;
    g.eps_mode = cfg->eps_mode;
    g.prec = cfg->precision;
    g.flux = cfg->flux;
    g.igm = cfg->equation == MR_EQ_EULER ? 1.0 / (cfg->phys[0] - 1.0) : 0.0;
    g.gcap = 0;
    long long off = 0, toff = 0;
    for (int l = g.lb; l <= g.L; ++l) {
        g.toff[l] = toff;
        const long long nl = 1LL << l;
        const int tx = g.d == 1 ? kTile1X : (g.d == 2 ? kTile2X : kTile3X);
        const int ty = g.d == 2 ? kTile2Y : kTile3Y;
        g.ntx[l] = (int)((nl + tx - 1) / tx);
        g.nty[l] = g.d >= 2 ? (int)((nl + ty - 1) / ty) : 1;
        g.ntz[l] = g.d == 3 ? (int)((nl + kTile3Z - 1) / kTile3Z) : 1;
        toff += (long long)g.ntx[l] * g.nty[l] * g.ntz[l];
        g.off[l] = off;
        g.N[l] = 1LL << (g.d * l);
        g.n[l] = 1 << l;
        for (int k = 0; k < 3; ++k) {
            g.dx[l][k] = (cfg->hi[k] - cfg->lo[k]) / g.n[l];
            g.rdx[l][k] = 1.0 / g.dx[l][k];
        }
        off += g.N[l];
    }
    h->ntot = off;
    h->reg = cfg->reflux && !g.gts;
    const size_t nd = (size_t)off * g.m;
    mr_status r = MR_OK;
    auto A = [&](mr_status s) {
        if (r == MR_OK) r = s;
    };
    A(dev_alloc(h, &g.st, off));
    A(dev_alloc(h, &g.flag, off));
    A(dev_alloc(h, &g.slot, off));
    A(dev_alloc(h, &g.ftop, 2));
    A(dev_alloc(h, &g.leaves, off));
    A(dev_alloc(h, &g.inner, off));
    A(dev_alloc(h, &g.counts, 3 * (LMAX + 1)));
    A(dev_alloc(h, &g.tflag, (size_t)toff));
    A(dev_alloc(h, &g.tlist, (size_t)toff));
    A(dev_alloc(h, &g.scale_bits, MMAX));
    A(dev_alloc(h, &g.dtp, 1));
    A(dev_alloc(h, &g.room, 4));
    A(dev_alloc(h, &g.err, 1));
    A(dev_alloc(h, &g.near, 1));
    A(dev_alloc(h, &g.wmax, 1));
    A(dev_alloc(h, &g.updates, 1));
    A(dev_alloc(h, &g.work, (LMAX + 1) * 4));
    A(dev_alloc(h, &h->d_bar, 2));
    A(dev_alloc(h, &h->d_nref, 1));
    if (r == MR_OK && !h->dry &&
        cudaMemsetAsync(g.work, 0, (LMAX + 1) * 4 * sizeof(unsigned long long), h->stream) != cudaSuccess)
        r = MR_E_CUDA; // cumulative counters: never cleared by mr_reset
    long long nblk = 0;
    for (int l = g.lb; l <= g.L; ++l) nblk += (g.N[l] + NTHREADS - 1) / NTHREADS;
    A(dev_alloc(h, &h->K.bc, 2 * nblk));
    A(dev_alloc(h, &h->d_part, (size_t)(LMAX + 1) * MASS_BLOCKS * g.m));
    (void)nd;
    h->fixed_bytes = h->bytes;
    // node arrays: the full tree of a new solver (every cell a node) plus the sink
    if (h->dry) {
        h->bytes += (size_t)(off + 1) * per_node_bytes(g, h->reg);
        g.cap = off + 1;
    } else if (r == MR_OK) {
        r = alloc_nodes(h, g, off + 1, h->node_allocs);
        h->bytes = h->fixed_bytes + (size_t)(off + 1) * per_node_bytes(g, h->reg);
    }
    if (r == MR_OK && !h->dry && !h->h_top) {
        if (cudaMallocHost((void**)&h->h_top, 4 * sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            r = MR_E_NOMEM;
        } else {
            memset(h->h_top, 0, 4 * sizeof(int));
        }
    }
    return r;
}

} // namespace

extern "C" {

mr_status mr_create(const mr_config* cfg, const double* q0, void* cuda_stream, mr_solver** out)
{
    if (!out) return MR_E_INVALID;
    *out = nullptr;
    if (validate(cfg) != MR_OK || !q0) return MR_E_INVALID;
    {
        // the exact footprint, projected before anything is allocated or read
        mr_solver probe;
        probe.dry = true;
        layout_alloc(&probe, cfg);
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess && probe.bytes > free_b + pool_cached_bytes()) {
            fprintf(stderr, "mr_create: needs %zu bytes of device memory, %zu free\n", probe.bytes, free_b);
            return MR_E_NOMEM;
        }
        cudaGetLastError();
    }
    mr_solver* h = new (std::nothrow) mr_solver();
    if (!h) return MR_E_NOMEM;
    h->cfg = *cfg;
    h->stream = (cudaStream_t)cuda_stream;
    h->K.st = h->stream;
    mr_status r = layout_alloc(h, cfg);
    if (r == MR_OK) r = init_state(h, q0);
    if (r != MR_OK) {
        fprintf(stderr, "mr_create: %s\n", h->err.c_str());
        mr_destroy(h);
        return r;
    }
    *out = h;
    return MR_OK;
}

mr_status mr_reset(mr_solver* h, const double* q0)
{
    if (!h || !q0) return MR_E_INVALID;
    return init_state(h, q0);
}

mr_status mr_set_tree(mr_solver* h, const unsigned char* lev)
{
    if (!h || !lev) return MR_E_INVALID;
    if (h->pos != 0) return MR_E_STATE;
    h->wmax_valid = false;
    Grid& g = h->K.g;
    const int L = g.L, lb = g.lb, d = g.d;
    std::vector<std::vector<uint8_t>> R(L + 1);
    for (int l = lb; l <= L; ++l) R[l].assign((size_t)g.N[l], 0);
    const long long NL = g.N[L], nL = g.n[L];
    auto coords = [&](int l, long long id, int c[3]) {
        const long long n = g.n[l];
        c[0] = (int)(id % n);
        c[1] = d > 1 ? (int)((id / n) % n) : 0;
        c[2] = d > 2 ? (int)(id / (n * n)) : 0;
    };
    auto lid = [&](int l, const int c[3]) {
        const long long n = g.n[l];
        return (long long)c[0] + n * ((long long)c[1] + n * (long long)c[2]);
    };
    (void)nL;
    for (long long id = 0; id < NL; ++id) {
        if (lev[id] < lb || lev[id] > L) {
            h->err = "set_tree: level out of range";
            return MR_E_INVALID;
        }
        int c[3];
        coords(L, id, c);
        for (int l = lb; l < lev[id]; ++l) {
            int p[3] = {c[0] >> (L - l), d > 1 ? c[1] >> (L - l) : 0, d > 2 ? c[2] >> (L - l) : 0};
            R[l][lid(l, p)] = 1;
        }
    }
    for (long long id = 0; id < NL; ++id) { // leaves partition the box as the map says
        int c[3];
        coords(L, id, c);
        int lv = lb;
        for (int l = lb; l < L; ++l) {
            int p[3] = {c[0] >> (L - l), d > 1 ? c[1] >> (L - l) : 0, d > 2 ? c[2] >> (L - l) : 0};
            if (!R[l][lid(l, p)]) break;
            lv = l + 1;
        }
        if (lv != lev[id]) {
            h->err = "set_tree: map is not a leaf partition";
            return MR_E_INVALID;
        }
    }
    for (int l = L - 1; l > lb; --l) // graded
        for (long long id = 0; id < g.N[l]; ++id) {
            if (!R[l][id]) continue;
            int c[3];
            coords(l, id, c);
            const int P[3] = {c[0] >> 1, c[1] >> 1, c[2] >> 1};
            for (int dz = (d > 2 ? -1 : 0); dz <= (d > 2 ? 1 : 0); ++dz)
                for (int dy = (d > 1 ? -1 : 0); dy <= (d > 1 ? 1 : 0); ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        const int off3[3] = {dx, dy, dz};
                        int q[3] = {0, 0, 0};
                        bool ok = true;
                        for (int k = 0; k < d; ++k) {
                            int p = P[k] + off3[k], n = g.n[l - 1];
                            if (g.bc[k] == MR_BC_PERIODIC) p = ((p % n) + n) % n;
                            else if (p < 0 || p >= n) ok = false;
                            q[k] = p;
                        }
                        if (ok && !R[l - 1][lid(l - 1, q)]) {
                            h->err = "set_tree: map is not graded";
                            return MR_E_INVALID;
                        }
                    }
        }
    h->K.leaf_copy(lb, L, F_QE, F_Q0);
    for (int l = L - 1; l >= lb; --l) h->K.project(l, PM_Q0);
    MR_CK(cudaMemsetAsync(g.flag, 0, h->ntot, h->stream));
    std::vector<uint8_t> fl((size_t)h->ntot, 0);
    for (int l = lb; l < L; ++l)
        for (long long id = 0; id < g.N[l]; ++id)
            if (R[l][id]) fl[g.off[l] + id] = FL_REF;
    MR_CK(cudaMemcpyAsync(g.flag, fl.data(), fl.size(), cudaMemcpyHostToDevice, h->stream));
    MR_TRY(set_capacity(h, h->ntot + 1, true)); // room for any tree, compacted at the end
    h->K.apply_tree(lb);
    h->K.compact(lb, L);
    for (int l = L - 1; l >= lb; --l) h->K.project(l, PM_Q0);
    h->K.leaf_copy(lb, L, F_Q0, F_QE);
    MR_TRY(sync_check(h));
    return fit_new_tree(h);
}

mr_status mr_create_from_state(const mr_config* cfg, long long n_leaves, const int* keys, const double* values,
                               double t, long long iters, void* cuda_stream, mr_solver** out)
{
    if (!out) return MR_E_INVALID;
    *out = nullptr;
    if (validate(cfg) != MR_OK || n_leaves < 1 || !keys || !values || !(t >= 0.0) || iters < 0)
        return MR_E_INVALID;
    const int d = cfg->dim, L = cfg->max_level, lb = cfg->min_level;
    const int m = cfg->equation == MR_EQ_EULER ? d + 2 : 1;
    if (iters % (1LL << (L - lb)) != 0) return MR_E_STATE; // not a macro-step boundary
    // finest-level leaf map: every finest cell covered by exactly one leaf
    const long long nL = 1LL << L, NL = 1LL << (d * L);
    std::vector<unsigned char> map((size_t)NL, 0xff);
    for (long long i = 0; i < n_leaves; ++i) {
        const int* K = keys + 4 * i;
        const int l = K[0];
        if (l < lb || l > L) return MR_E_INVALID;
        const long long span = 1LL << (L - l);
        long long lo3[3] = {0, 0, 0}, hi3[3] = {1, 1, 1};
        for (int k = 0; k < d; ++k) {
            if (K[1 + k] < 0 || K[1 + k] >= (1LL << l)) return MR_E_INVALID;
            lo3[k] = K[1 + k] * span;
            hi3[k] = lo3[k] + span;
        }
        for (long long z = lo3[2]; z < hi3[2]; ++z)
            for (long long y = lo3[1]; y < hi3[1]; ++y)
                for (long long x = lo3[0]; x < hi3[0]; ++x) {
                    unsigned char& c = map[(size_t)(x + nL * (y + nL * z))];
                    if (c != 0xff) return MR_E_INVALID; // overlapping leaves
                    c = (unsigned char)l;
                }
    }
    for (unsigned char c : map)
        if (c == 0xff) return MR_E_INVALID; // a hole in the partition
    // a solver on zero data without adaptation, then the saved tree and values
    mr_config c0 = *cfg;
    c0.adapt_mode = MR_ADAPT_NEVER;
    std::vector<double> zeros((size_t)m * NL, 0.0);
    mr_solver* h = nullptr;
    MR_TRY(mr_create(&c0, zeros.data(), cuda_stream, &h));
    h->cfg = *cfg;
    mr_status r = mr_set_tree(h, map.data());
    Grid& g = h->K.g;
    int* d_keys = nullptr;
    double* d_vals = nullptr;
    if (r == MR_OK) r = scratch(h, &d_keys, (size_t)4 * n_leaves);
    if (r == MR_OK) r = scratch(h, &d_vals, (size_t)m * n_leaves);
    if (r == MR_OK && cudaMemcpyAsync(d_keys, keys, sizeof(int) * 4 * (size_t)n_leaves, cudaMemcpyHostToDevice,
                                      h->stream) != cudaSuccess)
        r = MR_E_CUDA;
    if (r == MR_OK && cudaMemcpyAsync(d_vals, values, sizeof(double) * (size_t)m * n_leaves,
                                      cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
        r = MR_E_CUDA;
    if (r == MR_OK) {
        h->K.set_leaves(d_keys, d_vals, n_leaves);
        for (int l = L - 1; l >= lb; --l) h->K.project(l, PM_Q0);
        h->t = t;
        h->iters = iters;
        h->macros = iters >> (L - lb);
        h->pos = 0;
        r = sync_check(h);
    }
    if (d_keys) cudaFreeAsync(d_keys, h->stream);
    if (d_vals) cudaFreeAsync(d_vals, h->stream);
    (void)g;
    if (r != MR_OK) {
        mr_destroy(h);
        return r;
    }
    *out = h;
    return MR_OK;
}

mr_status mr_adapt(mr_solver* h)
{
    if (!h) return MR_E_INVALID;
    if (h->pos != 0) return MR_E_STATE;
    h->wmax_valid = false;
    Grid& g = h->K.g;
    MR_TRY(set_capacity(h, h->ntot + 1, true)); // room for any tree, compacted at the end
    h->K.leaf_copy(g.lb, g.L, F_QE, F_Q0);
    for (int l = g.L - 1; l >= g.lb; --l) h->K.project(l, PM_Q0);
    MR_TRY(adapt(h, g.lb));
    h->K.leaf_copy(g.lb, g.L, F_Q0, F_QE);
    MR_TRY(sync_check(h));
    return fit_new_tree(h);
}

mr_status mr_step(mr_solver* h, double t_target, long long* iters_out)
{
    if (!h) return MR_E_INVALID;
    if (h->pos != 0) return MR_E_STATE;
    const long long it0 = h->iters, nit = 1LL << (h->K.g.L - h->K.g.lb);
    while (h->t < t_target) {
        double dt;
        MR_TRY(head_enqueue(h)); // read back with the CFL speed
        MR_TRY(cfl_dt(h, &dt));
        if (h->h_top[2]) { // the macro step before halted: finish it, then this boundary again
            MR_TRY(recover(h));
            MR_TRY(run_iters(h, h->dt, 0));
            continue;
        }
        MR_TRY(head_finish(h));
        bool last = false;
        if (h->t + nit * dt >= t_target * (1.0 - 1e-14)) {
            dt = (t_target - h->t) / nit;
            last = true;
        }
        const double t0 = h->t;
        MR_TRY(run_iters(h, dt, nit));
        h->t = last ? t_target : t0 + nit * dt;
    }
    if (iters_out) *iters_out = h->iters - it0;
    return h->async ? MR_OK : sync_check(h);
}

mr_status mr_iterate(mr_solver* h, double dt, long long n, long long* iters_out)
{
    if (!h || !(dt > 0.0) || n < 0) return MR_E_INVALID;
    const long long it0 = h->iters, nit = 1LL << (h->K.g.L - h->K.g.lb);
    long long i = 0;
    while (i < n) { // whole macro steps at once (a graph), single iterations otherwise
        if (h->pos == 0) MR_TRY(boundary_check(h)); // capacity rule at the macro-step boundary
        const long long chunk = (h->pos == 0 && n - i >= nit) ? nit : 1;
        MR_TRY(run_iters(h, dt, chunk));
        for (long long k = 0; k < chunk; ++k) h->t += dt;
        i += chunk;
    }
    if (iters_out) *iters_out = h->iters - it0;
    return h->async ? MR_OK : sync_check(h);
}

mr_status mr_set_async(mr_solver* h, int enable)
{
    if (!h) return MR_E_INVALID;
    if (h->async_err && h->async_err != h->own_err) return MR_E_STATE; // a batch or server instance
    if (enable) {
        if (!h->own_err) {
            if (cudaMallocHost((void**)&h->own_err, sizeof(int)) != cudaSuccess) {
                cudaGetLastError();
                return MR_E_NOMEM;
            }
            *h->own_err = 0;
        }
        h->async_err = h->own_err;
        h->async = true;
        return MR_OK;
    }
    const mr_status r = mr_sync(h);
    h->async = false;
    h->async_err = nullptr;
    return r;
}

mr_status mr_set_grid_cap(mr_solver* h, int ctas)
{
    if (!h || ctas < 0) return MR_E_INVALID;
    if (h->K.g.gcap == ctas) return MR_OK;
    // a captured macro step holds the old launch shape: drop it once the
    // stream has passed it, and capture again at the next macro step
    if (h->macro_exec || h->head_exec) {
        MR_CK(cudaStreamSynchronize(h->stream));
        drop_graphs(h);
    }
    h->K.g.gcap = ctas;
    return MR_OK;
}

mr_status mr_reserve_nodes(mr_solver* h, long long nodes)
{
    if (!h || nodes < 0) return MR_E_INVALID;
    if (h->pos != 0) return MR_E_STATE;
    h->reserved = nodes;
    if (nodes + 1 <= h->K.g.cap) return MR_OK;
    MR_TRY(set_capacity(h, nodes + 1, true));
    return sync_check(h);
}

mr_status mr_set_launch_mode(mr_solver* h, int mode)
{
    if (!h || (mode != MR_LAUNCH_PERSISTENT && mode != MR_LAUNCH_GRAPH)) return MR_E_INVALID;
    if (h->pos != 0) return MR_E_STATE;
    // the macro-step kernel installs trees without a host check: room for every
    // cell first (the mode stays as it was if that fails)
    if (mode == MR_LAUNCH_PERSISTENT) {
        MR_TRY(set_capacity(h, h->ntot + 1, true));
        MR_TRY(sync_check(h));
    }
    h->launch_mode = mode;
    h->head_pending = h->head_done = false;
    return MR_OK;
}

mr_status mr_selftest_grid_wait(int ctas, int missing, double limit_s, void* cuda_stream)
{
    if (ctas < 1 || ctas > 1024 || missing < 0 || !(limit_s > 0.0) || limit_s > 60.0) return MR_E_INVALID;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    unsigned* bar = nullptr;
    if (cudaMalloc((void**)&bar, 4 * sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        return MR_E_NOMEM;
    }
    int* err = (int*)(bar + 2);
    int e = 0;
    mr_status r = MR_OK;
    if (cudaMemsetAsync(bar, 0, 4 * sizeof(unsigned), st) != cudaSuccess ||
        launch_grid_wait_test(st, ctas, missing, (unsigned long long)(limit_s * 1e9), bar, err) != 0 ||
        cudaMemcpyAsync(&e, err, sizeof e, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        r = MR_E_CUDA;
    else if (e & ERR_TIMEOUT)
        r = MR_E_TIMEOUT;
    cudaGetLastError();
    cudaFree(bar);
    return r;
}

mr_status mr_sync(mr_solver* h)
{
    if (!h) return MR_E_INVALID;
    MR_TRY(sync_check(h));
    if (h->async_err && *h->async_err) {
        h->err = "non-finite value found by a macro-step check";
        return MR_E_NUMERIC;
    }
    return MR_OK;
}

mr_status mr_read(mr_solver* h, int what, void* buf, size_t cap, size_t* used)
{
    if (!h) return MR_E_INVALID;
    Grid& g = h->K.g;
    const int m = g.m;
    int cnt[2 * (LMAX + 1)];
    MR_CK(cudaMemcpyAsync(cnt, g.counts, sizeof cnt, cudaMemcpyDeviceToHost, h->stream));
    MR_CK(cudaStreamSynchronize(h->stream));
    long long nleaf = 0, nnode = 0;
    for (int l = g.lb; l <= g.L; ++l) {
        nleaf += cnt[l];
        nnode += cnt[l] + cnt[LMAX + 1 + l];
    }
    size_t need;
    if (what == MR_READ_LEAF_KEYS) need = (size_t)nleaf * 4 * sizeof(int);
    else if (what == MR_READ_LEAF_VALUES) need = (size_t)nleaf * m * sizeof(double);
    else if (what == MR_READ_UNIFORM) need = (size_t)g.N[g.L] * m * sizeof(double);
    else if (what == MR_READ_STATS || what == MR_READ_PROFILE) need = 64 * sizeof(double);
    else return MR_E_INVALID;
    if (used) *used = need;
    if (!buf) return MR_OK;
    if (cap < need) return MR_E_INVALID;
    if (what == MR_READ_LEAF_KEYS || what == MR_READ_LEAF_VALUES) {
        unsigned char* tmp = nullptr; // transient
        MR_TRY(scratch(h, &tmp, need));
        int* keys = what == MR_READ_LEAF_KEYS ? (int*)tmp : nullptr;
        double* vals = what == MR_READ_LEAF_VALUES ? (double*)tmp : nullptr;
        long long base = 0;
        for (int l = g.lb; l <= g.L; ++l) {
            if (cnt[l]) h->K.pack(l, base, keys, vals);
            base += cnt[l];
        }
        if (need) MR_CK(cudaMemcpyAsync(buf, tmp, need, cudaMemcpyDeviceToHost, h->stream));
        MR_CK(cudaFreeAsync(tmp, h->stream));
    } else if (what == MR_READ_PROFILE) {
        double* P = (double*)buf;
        memset(P, 0, 64 * sizeof(double));
        unsigned long long w[(LMAX + 1) * 4];
        MR_CK(cudaMemcpyAsync(w, g.work, sizeof w, cudaMemcpyDeviceToHost, h->stream));
        MR_CK(cudaStreamSynchronize(h->stream));
        drain_events(h);
        P[0] = (double)h->prof_launches;
        P[1] = h->prof_ms;
        for (int l = 0; l <= LMAX; ++l)
            for (int s = 1; s <= 3; ++s) {
                P[1 + s] += (double)(w[l * 4 + s] - h->work0[l * 4 + s]);
                P[16 + l] += (double)w[l * 4 + s];
            }
        P[5] = (double)(h->K.n + h->stage_launches - h->prof_all0);
        for (int l = 0; l <= LMAX; ++l) P[40 + l] = h->prof_level_ms[l];
    } else if (what == MR_READ_UNIFORM) { // a transient pyramid for the inverse transform
        double* T = nullptr;
        uint8_t* us = nullptr;
        MR_TRY(scratch(h, &T, (size_t)h->ntot * m));
        MR_TRY(scratch(h, &us, (size_t)h->ntot));
        h->K.uniform(T, us);
        MR_CK(cudaMemcpyAsync(buf, T + g.off[g.L] * m, need, cudaMemcpyDeviceToHost, h->stream));
        MR_CK(cudaFreeAsync(T, h->stream));
        MR_CK(cudaFreeAsync(us, h->stream));
    } else {
        double* S = (double*)buf;
        memset(S, 0, 64 * sizeof(double));
        std::vector<double> part((size_t)(LMAX + 1) * MASS_BLOCKS * m, 0.0);
        for (int l = g.lb; l <= g.L; ++l) h->K.mass(l, h->d_part + (size_t)l * MASS_BLOCKS * m);
        MR_CK(cudaMemcpyAsync(part.data(), h->d_part, part.size() * sizeof(double), cudaMemcpyDeviceToHost,
                              h->stream));
        int ftop[2] = {0, 0};
        MR_CK(cudaMemcpyAsync(ftop, g.ftop, sizeof ftop, cudaMemcpyDeviceToHost, h->stream));
        unsigned long long near = 0, upd = 0;
        MR_CK(cudaMemcpyAsync(&near, g.near, sizeof near, cudaMemcpyDeviceToHost, h->stream));
        MR_CK(cudaMemcpyAsync(&upd, g.updates, sizeof upd, cudaMemcpyDeviceToHost, h->stream));
        MR_CK(cudaStreamSynchronize(h->stream));
        S[0] = h->t;
        S[1] = (double)h->iters;
        S[2] = (double)h->macros;
        S[3] = h->dt;
        S[4] = (double)nleaf;
        S[5] = (double)nnode;
        S[6] = (double)near;
        S[7] = (double)upd;
        S[61] = (double)h->halts;     // halted remeshes (node arrays grown mid macro step)
        S[62] = (double)ftop[0];      // free node slots
        S[13] = (double)(g.cap - 1);  // node slots
        S[14] = (double)h->bytes;     // device bytes held
        S[15] = (double)h->pos;
        for (int l = g.lb; l <= g.L; ++l) {
            S[16 + l] = cnt[l];
            double vol = 1.0;
            for (int k = 0; k < g.d; ++k) vol *= g.dx[l][k];
            for (int v = 0; v < m; ++v) {
                double s = 0.0;
                for (int b = 0; b < MASS_BLOCKS; ++b) s += part[((size_t)l * MASS_BLOCKS + b) * m + v];
                S[8 + v] += s * vol;
            }
        }
    }
    return sync_check(h);
}

mr_status mr_profile(mr_solver* h, int enable)
{
    if (!h) return MR_E_INVALID;
    if (enable) {
        if (h->ev.empty()) {
            h->ev.resize(2 * 4096);
            h->ev_level.assign(4096, 0);
            for (auto& e : h->ev) MR_CK(cudaEventCreate(&e));
        }
        if (!h->d_stamps) { // phase stamps of the macro-step kernel (not part of the footprint)
            const size_t b0 = h->bytes;
            MR_TRY(dev_alloc(h, &h->d_stamps, (size_t)2 * kStampCap));
            MR_TRY(dev_alloc(h, &h->d_nstamps, 1));
            h->bytes = b0;
        }
        MR_CK(cudaStreamSynchronize(h->stream));
        h->ev_used = 0;
        h->prof_ms = 0.0;
        for (double& x : h->prof_level_ms) x = 0.0;
        h->prof_launches = 0;
        h->prof_all0 = h->K.n + h->stage_launches;
        MR_CK(cudaMemcpyAsync(h->work0, h->K.g.work, sizeof h->work0, cudaMemcpyDeviceToHost, h->stream));
        MR_CK(cudaStreamSynchronize(h->stream));
        h->prof = true;
    } else {
        drain_events(h);
        h->prof = false;
    }
    return MR_OK;
}

void mr_destroy(mr_solver* h)
{
    if (!h) return;
    drop_graphs(h);
    if (h->h_top) {
        cudaStreamSynchronize(h->stream);
        cudaFreeHost(h->h_top);
    }
    for (void* p : h->node_allocs) cudaFreeAsync(p, h->stream);
    if (h->own_err) {
        cudaStreamSynchronize(h->stream); // the slot may still receive a pending copy
        cudaFreeHost(h->own_err);
    }
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    for (auto& e : h->ev) cudaEventDestroy(e);
    for (void* p : h->allocs) cudaFreeAsync(p, h->stream); // back to the pool, in stream order
    delete h;
}

const char* mr_last_error(const mr_solver* h) { return h ? h->err.c_str() : kNullErr; }

long long mr_launch_count(const mr_solver* h) { return h ? h->K.n + h->stage_launches : 0; }

mr_status mr_release_cached_memory(void)
{
    std::lock_guard<std::mutex> lock(g_pool_mutex);
    for (int dev = 0; dev < kMaxPoolDevices; ++dev)
        if (g_pool[dev] && cudaMemPoolTrimTo(g_pool[dev], 0) != cudaSuccess) {
            cudaGetLastError();
            return MR_E_CUDA;
        }
    return MR_OK;
}

} // extern "C"

// ---------------------------------------------------------------- progress
// Non-blocking progress of one problem toward t_target by whole macro steps.
// The CFL reduction of the next macro step is queued behind the current one,
// on the problem's own stream, with its value landing in *bits and an event
// recorded after it; once the event has fired, the host picks the step, the
// macro step (a graph) and the next CFL reduction are queued, and so on.  No
// call waits, so every problem runs at the pace of its own stream.
namespace {

// PG_SETTLE: the last macro step is queued, its halt record on the way
enum { PG_IDLE = 0, PG_WAIT = 1, PG_DONE = 2, PG_SETTLE = 3 };

struct Progress {
    int phase = PG_IDLE;
    mr_status status = MR_OK;
};

// queue the CFL reduction of the next macro step
mr_status progress_start(mr_solver* h, unsigned long long* bits, cudaEvent_t ev, Progress* pg)
{
    MR_TRY(head_enqueue(h));
    MR_TRY(cfl_enqueue(h, bits));
    MR_CK(cudaEventRecord(ev, h->stream));
    pg->phase = PG_WAIT;
    return MR_OK;
}

// the end of a problem's last macro step: its halt record read back before
// it counts as done
mr_status settle_start(mr_solver* h, cudaEvent_t ev, Progress* pg)
{
    MR_TRY(enqueue_slot_record(h));
    MR_CK(cudaEventRecord(ev, h->stream));
    pg->phase = PG_SETTLE;
    return MR_OK;
}

// one non-blocking attempt; returns true when the problem made progress
bool progress_poll(mr_solver* h, double t_target, unsigned long long* bits, const int* err, cudaEvent_t ev,
                   Progress* pg)
{
    if (pg->phase == PG_DONE) return false;
    if (pg->phase == PG_IDLE) {
        pg->status = progress_start(h, bits, ev, pg);
        if (pg->status != MR_OK) pg->phase = PG_DONE;
        return true;
    }
    const cudaError_t e = cudaEventQuery(ev);
    if (e == cudaErrorNotReady) return false;
    const bool settling = pg->phase == PG_SETTLE;
    pg->phase = PG_DONE;
    if (e != cudaSuccess) {
        pg->status = MR_E_CUDA;
        return true;
    }
    if (h->h_top[2]) { // a remesh of the previous macro step halted: finish it, then this boundary again
        pg->status = recover(h);
        if (pg->status == MR_OK) pg->status = run_iters(h, h->dt, 0);
        if (pg->status == MR_OK) pg->status = settling ? settle_start(h, ev, pg) : progress_start(h, bits, ev, pg);
        if (pg->status != MR_OK) pg->phase = PG_DONE;
        return true;
    }
    if (settling) return true; // done: its last macro step completed without a halt
    if (*err) { // the finiteness check of the previous macro step failed
        pg->status = sync_check(h);
        if (pg->status == MR_OK) pg->status = MR_E_NUMERIC;
        return true;
    }
    const long long nit = 1LL << (h->K.g.L - h->K.g.lb);
    pg->status = head_finish(h); // the head's count and the free-slot count arrived with the CFL value
    if (pg->status != MR_OK) return true;
    double dt = cfl_from_bits(h, *bits);
    bool last = false;
    if (h->t + nit * dt >= t_target * (1.0 - 1e-14)) {
        dt = (t_target - h->t) / nit;
        last = true;
    }
    const double t0 = h->t;
    pg->status = run_iters(h, dt, nit);
    h->t = last ? t_target : t0 + nit * dt;
    if (pg->status == MR_OK) {
        pg->status = last ? settle_start(h, ev, pg) : progress_start(h, bits, ev, pg);
        if (pg->status != MR_OK) pg->phase = PG_DONE;
    }
    return true;
}

// brief host pause when no problem could progress
void progress_pause()
{
    std::this_thread::sleep_for(std::chrono::microseconds(20));
}

} // namespace

// ---------------------------------------------------------------- batches
struct mr_batch {
    std::vector<mr_solver*> inst;
    std::vector<cudaStream_t> streams;  // one internal stream per instance
    std::vector<cudaEvent_t> ev;        // per instance: its CFL value has arrived
    cudaStream_t user = nullptr;
    cudaEvent_t join = nullptr;
    unsigned long long* bits = nullptr; // pinned: largest speed per instance
    int* errs = nullptr;                // pinned: device error bits per instance
    std::string err;
};

namespace {

void batch_free(mr_batch* b)
{
    for (mr_solver* h : b->inst) mr_destroy(h);
    for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
    for (cudaStream_t st : b->streams) cudaStreamDestroy(st);
    if (b->join) cudaEventDestroy(b->join);
    if (b->bits) cudaFreeHost(b->bits);
    if (b->errs) cudaFreeHost(b->errs);
    delete b;
}

mr_status batch_fail(mr_batch* b, int i, mr_status r)
{
    char buf[64];
    snprintf(buf, sizeof buf, "instance %d: ", i);
    b->err = std::string(buf) + (i >= 0 && i < (int)b->inst.size() ? b->inst[i]->err : std::string(""));
    return r;
}

} // namespace

extern "C" {

mr_status mr_batch_create(int n, const mr_config* cfgs, const double* const* q0s, void* cuda_stream,
                          mr_batch** out, int* failed_index)
{
    if (failed_index) *failed_index = -1;
    if (!out) return MR_E_INVALID;
    *out = nullptr;
    if (n < 1 || !cfgs || !q0s) return MR_E_INVALID;
    mr_batch* b = new (std::nothrow) mr_batch();
    if (!b) return MR_E_NOMEM;
    b->user = (cudaStream_t)cuda_stream;
    auto fail = [&](int i, mr_status r) {
        if (failed_index) *failed_index = i;
        batch_free(b);
        return r;
    };
    if (cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming) != cudaSuccess ||
        cudaMallocHost((void**)&b->bits, sizeof(unsigned long long) * n) != cudaSuccess ||
        cudaMallocHost((void**)&b->errs, sizeof(int) * n) != cudaSuccess) {
        cudaGetLastError();
        return fail(-1, MR_E_NOMEM);
    }
    memset(b->errs, 0, sizeof(int) * n);
    if (cudaEventRecord(b->join, b->user) != cudaSuccess) return fail(-1, MR_E_CUDA);
    for (int i = 0; i < n; ++i) {
        cudaStream_t st = nullptr;
        cudaEvent_t e = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return fail(i, MR_E_CUDA);
        b->streams.push_back(st);
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return fail(i, MR_E_CUDA);
        b->ev.push_back(e);
        if (cudaStreamWaitEvent(st, b->join, 0) != cudaSuccess) return fail(i, MR_E_CUDA);
        mr_solver* h = nullptr;
        const mr_status r = mr_create(&cfgs[i], q0s[i], st, &h);
        if (r != MR_OK) return fail(i, r);
        h->async_err = &b->errs[i];
        // instances run concurrently on their own streams: one kernel per
        // phase (captured graphs), since co-residency of several cooperative
        // grids is not something the instances could rely on
        h->launch_mode = MR_LAUNCH_GRAPH;
        b->inst.push_back(h);
    }
    *out = b;
    return MR_OK;
}

mr_status mr_batch_step(mr_batch* b, double t_target, long long* iters_out)
{
    if (!b) return MR_E_INVALID;
    const int n = (int)b->inst.size();
    for (int i = 0; i < n; ++i)
        if (b->inst[i]->pos != 0) return batch_fail(b, i, MR_E_STATE);
    long long it0 = 0;
    for (mr_solver* h : b->inst) it0 += h->iters;
    if (cudaEventRecord(b->join, b->user) != cudaSuccess) return MR_E_CUDA;
    std::vector<int> active;
    for (int i = 0; i < n; ++i) {
        if (cudaStreamWaitEvent(b->streams[i], b->join, 0) != cudaSuccess) return MR_E_CUDA;
        if (b->inst[i]->t < t_target) active.push_back(i);
    }
    // every instance progresses at its own pace (see progress_poll)
    std::vector<Progress> pg(n);
    for (int i = 0; i < n; ++i)
        if (b->inst[i]->t >= t_target) pg[i].phase = PG_DONE;
    for (;;) {
        bool busy = false, moved = false;
        for (int i : active) {
            if (pg[i].phase == PG_DONE) continue;
            moved |= progress_poll(b->inst[i], t_target, &b->bits[i], &b->errs[i], b->ev[i], &pg[i]);
            if (pg[i].phase == PG_DONE && pg[i].status != MR_OK) return batch_fail(b, i, pg[i].status);
            busy |= pg[i].phase != PG_DONE;
        }
        if (!busy) break;
        if (!moved) progress_pause();
    }
    long long it1 = 0;
    for (int i = 0; i < n; ++i) {
        mr_solver* h = b->inst[i];
        const mr_status r = sync_check(h);
        if (r != MR_OK) return batch_fail(b, i, r);
        if (b->errs[i]) return batch_fail(b, i, MR_E_NUMERIC);
        it1 += h->iters;
    }
    if (iters_out) *iters_out = it1 - it0;
    return MR_OK;
}

mr_status mr_batch_set_grid_cap(mr_batch* b, int ctas)
{
    if (!b || ctas < 0) return MR_E_INVALID;
    for (int i = 0; i < (int)b->inst.size(); ++i) {
        const mr_status r = mr_set_grid_cap(b->inst[i], ctas);
        if (r != MR_OK) return batch_fail(b, i, r);
    }
    return MR_OK;
}

mr_solver* mr_batch_instance(mr_batch* b, int i)
{
    return (b && i >= 0 && i < (int)b->inst.size()) ? b->inst[i] : nullptr;
}

const char* mr_batch_last_error(const mr_batch* b) { return b ? b->err.c_str() : kNullErr; }

void mr_batch_destroy(mr_batch* b)
{
    if (b) batch_free(b);
}

} // extern "C"

// ---------------------------------------------------------------- serving
// A request: one problem with its own end time.  State: queued -> active
// (admitted, advancing one macro step per round) -> finishing (last macro
// step enqueued) -> done (its stream reached the end; result readable).
struct mr_request {
    long long id = 0;
    mr_config cfg{};
    std::vector<double> q0;
    double t_end = 0.0;
    size_t proj = 0;        // projected device footprint
    size_t bytes = 0;       // charged: the larger of proj and the solver's footprint
    int slot = -1;          // pinned host slot while admitted
    mr_solver* h = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;   // CFL value has arrived
    cudaEvent_t fin = nullptr;  // all work of the request has completed
    int state = 0;              // 0 queued, 1 active, 2 finishing, 3 done
    mr_status status = MR_OK;
    Progress pg;
};

struct mr_server {
    size_t budget = 0, used = 0;
    int max_active = 0;
    cudaStream_t user = nullptr;
    long long next_id = 1;
    std::vector<mr_request*> queue, active, finishing;
    std::vector<long long> completed;  // finished, not yet reported by poll
    std::vector<mr_request*> all;      // every request not yet released
    unsigned long long* bits = nullptr; // pinned [max_active]
    int* errs = nullptr;                // pinned [max_active]
    std::vector<int> free_slots;
    int gcap = 0;                       // stage-launch block cap of admitted solvers
    std::string err;
};

namespace {

void request_free(mr_server* s, mr_request* q)
{
    if (q->h) mr_destroy(q->h);
    if (q->ev) cudaEventDestroy(q->ev);
    if (q->fin) cudaEventDestroy(q->fin);
    if (q->st) cudaStreamDestroy(q->st);
    if (q->slot >= 0) s->free_slots.push_back(q->slot);
    if (q->state == 1 || q->state == 2 || (q->state == 3 && q->h)) s->used -= q->bytes;
    delete q;
}

mr_request* find_request(mr_server* s, long long id)
{
    for (mr_request* q : s->all)
        if (q->id == id) return q;
    return nullptr;
}

// Projected device bytes of a configuration while it runs: the per-cell
// arrays, plus node arrays for the projected node count at the capacity rule.
// Projected nodes: an adapted tree concentrates on fronts of codimension one,
// about kFrontWidth nodes per finest cell of a (d-1)-dimensional slice, i.e.
// min(all cells, kFrontWidth 2^{(d-1) L}).  (Creating the solver briefly needs
// the full tree; mr_create checks that against the free memory.)
constexpr long long kFrontWidth = 64;

size_t projected_bytes(const mr_config* cfg)
{
    mr_solver probe;
    probe.dry = true;
    probe.cfg = *cfg;
    layout_alloc(&probe, cfg);
    long long nodes = kFrontWidth << ((cfg->dim - 1) * cfg->max_level);
    if (nodes > probe.ntot) nodes = probe.ntot;
    long long slots = nodes + 2 * (nodes / 4 > kMinSlots ? nodes / 4 : kMinSlots) + 1; // the capacity rule
    if (slots > probe.ntot + 1) slots = probe.ntot + 1;
    return probe.fixed_bytes + (size_t)slots * per_node_bytes(probe.K.g, probe.reg);
}

// admit queued requests in arrival order while the budget and the slot
// count allow; a request that fails to start is completed with its status
mr_status admit(mr_server* s)
{
    size_t k = 0;
    while (k < s->queue.size()) {
        mr_request* q = s->queue[k];
        if ((int)s->active.size() + (int)s->finishing.size() >= s->max_active || s->free_slots.empty() ||
            s->used + q->bytes > s->budget)
            break; // first come, first served: later requests wait too
        q->slot = s->free_slots.back();
        s->free_slots.pop_back();
        s->errs[q->slot] = 0;
        mr_status r = MR_OK;
        if (cudaStreamCreateWithFlags(&q->st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&q->ev, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&q->fin, cudaEventDisableTiming) != cudaSuccess)
            r = MR_E_CUDA;
        if (r == MR_OK) r = mr_create(&q->cfg, q->q0.data(), q->st, &q->h);
        q->q0.clear();
        q->q0.shrink_to_fit();
        ++k;
        if (r != MR_OK) {
            s->free_slots.push_back(q->slot);
            q->slot = -1;
            q->status = r;
            q->state = 3;
            s->completed.push_back(q->id);
            continue;
        }
        q->h->async_err = &s->errs[q->slot];
        q->h->launch_mode = MR_LAUNCH_GRAPH; // concurrent requests: as batch instances
        if (s->gcap) mr_set_grid_cap(q->h, s->gcap); // nothing captured yet: cannot fail
        q->bytes = q->h->bytes > q->proj ? q->h->bytes : q->proj; // a new tree holds room for every cell
        s->used += q->bytes;
        q->state = q->h->t < q->t_end ? 1 : 2;
        if (q->state == 1) s->active.push_back(q);
        else {
            cudaEventRecord(q->fin, q->st);
            s->finishing.push_back(q);
        }
    }
    s->queue.erase(s->queue.begin(), s->queue.begin() + k);
    return MR_OK;
}

// move finished requests whose stream has drained to the completed list
void reap(mr_server* s)
{
    std::vector<mr_request*> keep;
    for (mr_request* q : s->finishing) {
        const cudaError_t e = cudaEventQuery(q->fin);
        if (e == cudaErrorNotReady) {
            keep.push_back(q);
            continue;
        }
        if (q->status == MR_OK) q->status = e != cudaSuccess ? MR_E_CUDA : sync_check(q->h);
        if (q->status == MR_OK && s->errs[q->slot]) q->status = MR_E_NUMERIC;
        s->free_slots.push_back(q->slot);
        q->slot = -1;
        q->state = 3;
        s->completed.push_back(q->id);
    }
    s->finishing.swap(keep);
}

} // namespace

extern "C" {

mr_status mr_server_create(size_t mem_budget_bytes, int max_active, void* cuda_stream, mr_server** out)
{
    if (!out) return MR_E_INVALID;
    *out = nullptr;
    if (max_active < 1 || mem_budget_bytes == 0) return MR_E_INVALID;
    mr_server* s = new (std::nothrow) mr_server();
    if (!s) return MR_E_NOMEM;
    s->budget = mem_budget_bytes;
    s->max_active = max_active;
    s->user = (cudaStream_t)cuda_stream;
    if (cudaMallocHost((void**)&s->bits, sizeof(unsigned long long) * max_active) != cudaSuccess ||
        cudaMallocHost((void**)&s->errs, sizeof(int) * max_active) != cudaSuccess) {
        cudaGetLastError();
        if (s->bits) cudaFreeHost(s->bits);
        delete s;
        return MR_E_NOMEM;
    }
    for (int i = max_active - 1; i >= 0; --i) s->free_slots.push_back(i);
    *out = s;
    return MR_OK;
}

mr_status mr_server_set_grid_cap(mr_server* s, int ctas)
{
    if (!s || ctas < 0) return MR_E_INVALID;
    s->gcap = ctas;
    return MR_OK;
}

mr_status mr_server_submit(mr_server* s, const mr_config* cfg, const double* q0, double t_end, long long* id)
{
    if (!s || !cfg || !q0 || !id || !(t_end >= 0.0)) return MR_E_INVALID;
    if (validate(cfg) != MR_OK) {
        s->err = "submit: invalid configuration";
        return MR_E_INVALID;
    }
    mr_request* q = new (std::nothrow) mr_request();
    if (!q) return MR_E_NOMEM;
    q->cfg = *cfg;
    q->t_end = t_end;
    q->bytes = q->proj = projected_bytes(cfg);
    if (q->bytes > s->budget) {
        delete q;
        s->err = "submit: the request alone exceeds the memory budget";
        return MR_E_NOMEM;
    }
    const int m = cfg->equation == MR_EQ_EULER ? cfg->dim + 2 : 1;
    const size_t n = (size_t)m << (cfg->dim * cfg->max_level);
    q->q0.assign(q0, q0 + n);
    q->id = s->next_id++;
    s->queue.push_back(q);
    s->all.push_back(q);
    *id = q->id;
    return MR_OK;
}

mr_status mr_server_advance(mr_server* s, int* n_active, int* n_queued)
{
    if (!s) return MR_E_INVALID;
    reap(s);
    MR_TRY(admit(s));
    // every active request whose previous macro step has completed queues
    // its next one (see progress_poll); nothing here waits
    std::vector<mr_request*> still;
    for (mr_request* q : s->active) {
        progress_poll(q->h, q->t_end, &s->bits[q->slot], &s->errs[q->slot], q->ev, &q->pg);
        const size_t charge = q->h->bytes > q->proj ? q->h->bytes : q->proj; // after a resize of its node arrays
        s->used += charge;
        s->used -= q->bytes;
        q->bytes = charge;
        if (q->pg.phase == PG_DONE) {
            q->status = q->pg.status;
            cudaEventRecord(q->fin, q->st);
            q->state = 2;
            s->finishing.push_back(q);
        } else {
            still.push_back(q);
        }
    }
    s->active.swap(still);
    reap(s);
    if (n_active) *n_active = (int)(s->active.size() + s->finishing.size());
    if (n_queued) *n_queued = (int)s->queue.size();
    return MR_OK;
}

mr_status mr_server_poll(mr_server* s, long long* ids, int cap, int* n_done)
{
    if (!s || !n_done || (cap > 0 && !ids)) return MR_E_INVALID;
    reap(s);
    const int n = (int)s->completed.size() < cap ? (int)s->completed.size() : cap;
    for (int i = 0; i < n; ++i) ids[i] = s->completed[i];
    s->completed.erase(s->completed.begin(), s->completed.begin() + n);
    *n_done = n;
    return MR_OK;
}

mr_status mr_server_status(mr_server* s, long long id)
{
    if (!s) return MR_E_INVALID;
    mr_request* q = find_request(s, id);
    if (!q) return MR_E_INVALID;
    return q->state == 3 ? q->status : MR_E_STATE;
}

mr_solver* mr_server_result(mr_server* s, long long id)
{
    if (!s) return nullptr;
    mr_request* q = find_request(s, id);
    return (q && q->state == 3) ? q->h : nullptr;
}

mr_status mr_server_release(mr_server* s, long long id)
{
    if (!s) return MR_E_INVALID;
    for (size_t i = 0; i < s->all.size(); ++i) {
        mr_request* q = s->all[i];
        if (q->id != id) continue;
        if (q->state != 3) return MR_E_STATE;
        s->all.erase(s->all.begin() + i);
        request_free(s, q);
        return MR_OK;
    }
    return MR_E_INVALID;
}

size_t mr_server_memory(const mr_server* s) { return s ? s->used : 0; }

const char* mr_server_last_error(const mr_server* s) { return s ? s->err.c_str() : kNullErr; }

void mr_server_destroy(mr_server* s)
{
    if (!s) return;
    for (mr_request* q : s->finishing) cudaEventSynchronize(q->fin);
    for (mr_request* q : s->all) request_free(s, q);
    if (s->bits) cudaFreeHost(s->bits);
    if (s->errs) cudaFreeHost(s->errs);
    delete s;
}

} // extern "C"

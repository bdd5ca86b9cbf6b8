// Machinery shared by the pair kernels (gather and Newton-III symmetric):
// force-law constants, kernel arguments, mbarrier and bulk-copy helpers,
// the per-warp staging ring, compensated accumulation, and the host-side
// argument checks and workspace layout.  Included by one translation unit
// per kernel family (internal linkage: each gets its own copy).
#pragma once

#include <math.h>

#include "hacc_common.cuh"

namespace hacc {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr long long WAIT_LIMIT_CYCLES = 2000000000LL;  // default wait bound: ~1 s at 2 GHz
constexpr uint32_t WAIT_HINT_NS = 100000;  // a waiting warp may sleep up to 0.1 ms per try

// FORCE: accelerations.  ADJOINT: dL/dx.  ADJOINT_GM: dL/dx and dL/dm.
// POTENTIAL: the short-range potential of each particle.
enum Mode { FORCE = 0, ADJOINT = 1, ADJOINT_GM = 2, POTENTIAL = 3 };

__host__ __device__ constexpr bool is_adjoint(int mode) { return mode == ADJOINT || mode == ADJOINT_GM; }

struct PairConsts {
    float eps;      // softening
    float rc2e;     // r_c^2 + eps (cut on se = s + eps)
    float nc[6];    // -(coefficients of poly~ in se), for f
    float kp[5];    // -2 (k+1) c~_{k+1}: Horner coefficients of -2 poly~'(se)
    float pv[7];    // pair potential V = pv(se) - (se)^-1/2: degree-6 coefficients in se
};

struct KArgs {
    const hacc_volume *vols;
    const int32_t *cell_start;
    const int64_t *nbr_off;
    const int32_t *nbr_cell;
    const int8_t *nbr_shift;
    const int4 *tasks;
    const int32_t *order;  // task_order: heaviest first
    const int32_t *n_tasks;
    const float4 *origin;  // per cell (leaf) origin, or NULL: chaining-mesh cell c sits at c w
    const float4 *pos;   // sorted (ox, oy, oz, m)
    const float4 *lam;   // sorted (lx, ly, lz, 0), adjoint only
    const int32_t *perm;
    float *out_x, *out_y, *out_z, *out_m;
    int32_t *counter;
    uint32_t *status;
    PairConsts k;
    const uint32_t *mass_varies;  // 0: every mass equal (the equal-mass force paths); NULL: general
    long long wait_limit;         // bound of each tile wait, clock64 cycles
    // sizes the debug build's bounds checks compare indices with
    int64_t N, n_cells, n_entries, task_cap;
    int V;
};

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ uint32_t mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(WAIT_HINT_NS)
        : "memory");
    return ok;
}

// Lane 0 only: pieces of a multi-segment tile.  Each bulk copy first raises
// the barrier's expected byte count; one arrive after the last copy ends the
// tile, so the phase cannot complete before every copy was issued.
__device__ __forceinline__ void tma_expect_copy(uint32_t bar, uint32_t dst, const void *src, uint32_t bytes)
{
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// All lanes wait for a barrier phase; false (uniformly) once the wait has
// lasted `limit` clock64 cycles of lane 0, checked before every poll.
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, long long limit)
{
    const long long t0 = clock64();
    while (true) {
        const int late = (clock64() - t0) >= limit;
        if (__shfl_sync(FULL, late, 0)) return false;
        const uint32_t ok = mbar_try_wait(bar, parity);
        if (__all_sync(FULL, ok)) return true;
    }
}

// The number of tasks to run, and task t of the heaviest-first order, with
// whether it may be run.  A product build just reads them.  A debug build
// (HACC_DEBUG_BOUNDS) first checks every index the task leads to -- the task
// count against the task buffer, its order entry and record, its volume, and
// on a chaining mesh its cell, its slot range and each entry of the cell's
// neighbour list with the slot range that entry names -- and skips a task
// that fails with HACC_STATUS_BOUNDS set, so that corrupted lists or tasks
// never turn into out-of-range accesses.  (Tree lists are checked up to the
// volume: the leaf count lives on the device.)  Warp-uniform.
__device__ __forceinline__ int task_count(const KArgs &a)
{
    const int nt = *a.n_tasks;
#ifdef HACC_DEBUG_BOUNDS
    if (nt < 0 || nt > a.task_cap) {
        if ((threadIdx.x & 31) == 0) atomicOr(a.status, HACC_STATUS_BOUNDS);
        return nt < 0 ? 0 : (int)a.task_cap;
    }
#endif
    return nt;
}

__device__ __forceinline__ bool take_task(const KArgs &a, int t, int lane, int4 &task, const int32_t *order)
{
#ifndef HACC_DEBUG_BOUNDS
    task = a.tasks[order ? order[t] : t];
    return true;
#else
    const int oi = order ? order[t] : t;
    bool ok = oi >= 0 && oi < a.task_cap;
    task = ok ? a.tasks[oi] : make_int4(0, 0, 0, 0);
    ok = ok && task.w >= 0 && task.w < a.V;
    if (ok && !a.origin) {
        const hacc_volume &vol = a.vols[task.w];
        const int64_t cb = vol.cell_base, ce = vol.cell_base + (int64_t)vol.n * vol.n * vol.n;
        ok = task.x >= cb && task.x < ce && ce <= a.n_cells;
        if (ok) {
            const int s0 = a.cell_start[task.x], s1 = a.cell_start[task.x + 1];
            ok = 0 <= s0 && s0 <= task.y && task.y < task.z && task.z <= s1 && s1 <= a.N;
        }
        if (ok) {
            const int64_t e0 = a.nbr_off[task.x], e1 = a.nbr_off[task.x + 1];
            ok = e0 >= 0 && e1 == e0 + vol.S && e1 <= a.n_entries;
            if (ok) {
                bool lane_ok = true;
                for (int64_t e = e0 + lane; e < e1; e += 32) {
                    const int cp = a.nbr_cell[e];
                    const int sh = a.nbr_shift[e];
                    bool eok = cp >= cb && cp < ce && sh >= 0 && sh < 27;
                    if (eok) {
                        const int j0 = a.cell_start[cp], j1 = a.cell_start[cp + 1];
                        eok = 0 <= j0 && j0 <= j1 && j1 <= a.N;
                    }
                    lane_ok = lane_ok && eok;
                }
                ok = __all_sync(FULL, lane_ok);
            }
        }
    }
    ok = __all_sync(FULL, ok);
    if (!ok && lane == 0) atomicOr(a.status, HACC_STATUS_BOUNDS);
    return ok;
#endif
}

// s = a + b exactly as s + err (Knuth's TwoSum), err added to the low word.
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float b)
{
    float s = __fadd_rn(hi, b);
    float bp = __fsub_rn(s, hi);
    float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(b, bp));
    hi = s;
    lo = __fadd_rn(lo, err);
}


// Hardware reciprocal square root (MUFU) without the denormal-input fix-up
// that rsqrtf() adds: its argument s + eps is at least eps, a normal float.
__device__ __forceinline__ float rsqrt_hw(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Adjoint accumulator layout (sizes the adjoint's shared memory): room for
// two i per lane with eight sums each (four i with the W form's three fit).
constexpr int ADJ_NACC = 8;
constexpr int ADJ_IPL_MAX = 2;
constexpr int ADJ_COMP_BYTES = ADJ_IPL_MAX * ADJ_NACC * 2 * 32 * 4;

// Adjoint accumulators per i particle: U (3) = sum f lam_j, V = sum m_j f,
// X (3) = sum fp2 (m_i d.lam_j - m_j d.lam_i) d, G = sum f d.lam_j (with dL/dm
// only).  Without dL/dm (the W form) the three sums collapse into one
// vector: with mu = m_i lam_j - m_j lam_i, W (3) = sum f mu + fp2 (d.mu) d =
// dL/dx_i (equal masses: mu / m summed, dL/dx_i = m W).  Float32 partial sums
// live in registers for one tile; the compensated (hi, lo) totals live in
// shared memory, lane-contiguous, so that two i particles per lane fit the
// register budget.
__host__ __device__ constexpr bool adj_wform(int mode) { return mode == ADJOINT; }
__host__ __device__ constexpr int adj_nacc(int mode) { return mode == ADJOINT_GM ? 8 : (adj_wform(mode) ? 3 : 7); }

template <int MODE, int IPL, int NC = adj_nacc(MODE)>
struct AccAdj {
    static constexpr int NACC = NC;
    static_assert(IPL * NC <= ADJ_IPL_MAX * ADJ_NACC, "compensated sums exceed the shared-memory slots");
    float p[IPL][ADJ_NACC];
    float *comp;  // [IPL][NACC][hi, lo][32 lanes]
    int lane;
    __device__ __forceinline__ float &hi(int u, int k) const { return comp[((u * NACC + k) * 2 + 0) * 32 + lane]; }
    __device__ __forceinline__ float &lo(int u, int k) const { return comp[((u * NACC + k) * 2 + 1) * 32 + lane]; }
    __device__ __forceinline__ AccAdj(float *c, int ln) : comp(c), lane(ln)
    {
#pragma unroll
        for (int u = 0; u < IPL; ++u)
#pragma unroll
            for (int k = 0; k < ADJ_NACC; ++k) p[u][k] = 0.f;
#pragma unroll
        for (int u = 0; u < IPL; ++u)
#pragma unroll
            for (int k = 0; k < NACC; ++k) hi(u, k) = lo(u, k) = 0.f;
    }
    __device__ __forceinline__ void fold()
    {
#pragma unroll
        for (int u = 0; u < IPL; ++u)
#pragma unroll
            for (int k = 0; k < NACC; ++k) {
                float h = hi(u, k), l = lo(u, k);
                two_sum_acc(h, l, p[u][k]);
                hi(u, k) = h;
                lo(u, k) = l;
                p[u][k] = 0.f;
            }
    }
    __device__ __forceinline__ float total(int u, int k) const { return hi(u, k) + lo(u, k); }
};


// Sorted cotangent records (lx, ly, lz, 0) for the adjoint.
__global__ void __launch_bounds__(256)
k_gather_lam(int64_t N, const int32_t *__restrict__ perm, const float *__restrict__ gx,
             const float *__restrict__ gy, const float *__restrict__ gz, float4 *__restrict__ lam)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N;
         k += (int64_t)gridDim.x * blockDim.x) {
        int i = perm[k];
        lam[k] = make_float4(gx[i], gy[i], gz[i], 0.f);
    }
}

// Shared memory of one warp: STAGES tiles (two arrays in the adjoint),
// STAGES mbarriers and, in the adjoint, the compensated totals; padded so
// that every warp's tiles start 128-B aligned.
__host__ __device__ constexpr int warp_tiles_bytes(int mode, int jt, int stages)
{
    return stages * (is_adjoint(mode) ? 2 : 1) * jt * 16;
}

__host__ __device__ constexpr int warp_smem_bytes(int mode, int jt, int stages)
{
    return ((warp_tiles_bytes(mode, jt, stages) + stages * 8 + (is_adjoint(mode) ? ADJ_COMP_BYTES : 0)) + 127) / 128 *
           128;
}

// Per-warp staging ring: STAGES tiles, their mbarriers and the lifetime tile
// counters (tile t lives in stage t % STAGES, phase parity (t / STAGES) & 1).
template <int MODE, int JT, int STAGES>
struct Ring {
    static constexpr int NBUF = is_adjoint(MODE) ? 2 : 1;
    float4 *tiles;
    uint64_t *bars;
    uint32_t issued = 0, consumed = 0;
    __device__ __forceinline__ float4 *tile(uint32_t st) const { return tiles + (size_t)st * NBUF * JT; }
    __device__ __forceinline__ uint32_t bar(uint32_t st) const { return smem_addr(&bars[st]); }
    // Stage the next tile: consecutive pieces of the group's entries (entry
    // counts in lane k's `cnt`, first records in lane k's `jb`) until JT
    // records or the group is exhausted, one bulk copy per piece (plus the
    // cotangents in the adjoint).  Warp-uniform; false if nothing was left.
    __device__ __forceinline__ bool produce(const KArgs &a, int lane, int ng, int cnt, int jb, int &k, int &off)
    {
        const uint32_t st = issued % STAGES;
        float4 *dst = tile(st);
        int filled = 0;
        bool fenced = false;
        while (k < ng && filled < JT) {
            const int c = __shfl_sync(FULL, cnt, k);
            if (off >= c) {
                ++k;
                off = 0;
                continue;
            }
            const int n = min(JT - filled, c - off);
            const int src = __shfl_sync(FULL, jb, k) + off;
            if (lane == 0) {
                if (!fenced) {
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    fenced = true;
                }
                tma_expect_copy(bar(st), smem_addr(dst + filled), a.pos + src, (uint32_t)n * 16u);
                if constexpr (NBUF == 2)
                    tma_expect_copy(bar(st), smem_addr(dst + JT + filled), a.lam + src, (uint32_t)n * 16u);
            }
            filled += n;
            off += n;
        }
        if (filled == 0) return false;
        if (lane == 0) mbar_arrive(bar(st));
        ++issued;
        return true;
    }
    // bounded wait for the next tile; false if the wait ran out
    __device__ __forceinline__ bool wait_next(long long limit) const
    {
        const uint32_t st = consumed % STAGES;
        return warp_wait(bar(st), (consumed / STAGES) & 1u, limit);
    }
    // after a timeout: let the copies still in flight land before leaving, each
    // wait bounded by the default limit whatever bound gave up
    __device__ __forceinline__ void drain()
    {
        while (consumed < issued) {
            warp_wait(bar(consumed % STAGES), (consumed / STAGES) & 1u, WAIT_LIMIT_CYCLES);
            ++consumed;
        }
    }
};

// poly~(se) = poly(se - eps): c~_m = sum_{k>=m} c_k C(k, m) (-eps)^(k-m), in float64.
void pair_consts(const hacc_sr_params *p, PairConsts &K)
{
    double c[6], ct[6];
    for (int k = 0; k < 6; ++k) c[k] = (double)p->c[k];
    const double e = -(double)p->eps;
    const double binom[6][6] = {{1, 0, 0, 0, 0, 0},  {1, 1, 0, 0, 0, 0},   {1, 2, 1, 0, 0, 0},
                                {1, 3, 3, 1, 0, 0},  {1, 4, 6, 4, 1, 0},   {1, 5, 10, 10, 5, 1}};
    for (int mdeg = 0; mdeg < 6; ++mdeg) {
        double s = 0.0;
        for (int k = mdeg; k < 6; ++k) s += c[k] * binom[k][mdeg] * pow(e, (double)(k - mdeg));
        ct[mdeg] = s;
    }
    K.eps = p->eps;
    K.rc2e = (float)((double)p->rcut * (double)p->rcut + (double)p->eps);
    for (int k = 0; k < 6; ++k) K.nc[k] = (float)(-ct[k]);
    for (int k = 0; k < 5; ++k) K.kp[k] = (float)(-2.0 * (k + 1) * ct[k + 1]);
    // potential: V(s) = C0 - (s + eps)^-1/2 - P(s) / 2 with P(s) = sum_k c_k s^(k+1) / (k+1),
    // C0 = (rc^2 + eps)^-1/2 + P(rc^2) / 2 so that V(rc^2) = 0; expanded in se = s + eps
    double Pm[7] = {0, 0, 0, 0, 0, 0, 0};  // P(s) = sum_m Pm[m] s^m
    for (int k = 0; k < 6; ++k) Pm[k + 1] = c[k] / (double)(k + 1);
    const double rc2 = (double)p->rcut * (double)p->rcut;
    double Prc = 0.0;
    for (int mdeg = 6; mdeg >= 1; --mdeg) Prc = (Prc + Pm[mdeg]) * rc2;
    const double C0 = 1.0 / sqrt(rc2 + (double)p->eps) + 0.5 * Prc;
    for (int jdeg = 0; jdeg <= 6; ++jdeg) {
        double acc = 0.0;
        for (int mdeg = jdeg; mdeg <= 6; ++mdeg) {
            double bin = 1.0;  // C(mdeg, jdeg)
            for (int q = 0; q < jdeg; ++q) bin = bin * (double)(mdeg - q) / (double)(q + 1);
            acc += -0.5 * Pm[mdeg] * bin * pow(e, (double)(mdeg - jdeg));
        }
        K.pv[jdeg] = (float)(acc + (jdeg == 0 ? C0 : 0.0));
    }
}

// Workspace of the pair calls: the task counter, the adjoints' sorted
// cotangents (16 B per particle), and the symmetric kernels' float64 sums
// (3 per particle for the force, 8 for the adjoint).
constexpr int SYM_ACC_MAX = 8;

struct ForceWs {
    int32_t *counter;
    float4 *lam;
    double *acc;
    size_t total;
};

ForceWs force_layout(const hacc_mesh *mesh, void *ws)
{
    ForceWs F{};
    char *p = reinterpret_cast<char *>(ws);
    const size_t lam_bytes = round_up((size_t)mesh->N * 16, 256);
    F.counter = reinterpret_cast<int32_t *>(p);
    F.lam = reinterpret_cast<float4 *>(p ? p + 256 : nullptr);
    F.acc = reinterpret_cast<double *>(p ? p + 256 + lam_bytes : nullptr);
    F.total = 256 + lam_bytes + round_up((size_t)mesh->N * 8 * SYM_ACC_MAX, 256);
    return F;
}

int check_common(const hacc_mesh *mesh, const hacc_binned *b, const hacc_lists *l, const hacc_sr_params *p,
                 const hacc_launch *launch, void *ws, size_t ws_bytes, uint32_t *status)
{
    if (!mesh || !b || !l || !p || !mesh->vols || !status || !ws || !aligned16(ws)) return HACC_ERR_INVALID;
    if (!(p->eps > 0.0f) || !isfinite(p->eps) || !(p->rcut > 0.0f) || !isfinite(p->rcut)) return HACC_ERR_INVALID;
    for (int k = 0; k < 6; ++k)
        if (!isfinite(p->c[k])) return HACC_ERR_INVALID;
    if (!b->cell_start) return HACC_ERR_INVALID;
    if (mesh->N > 0 && (!b->perm || !b->sorted4 || !aligned16(b->sorted4))) return HACC_ERR_INVALID;
    if (!l->nbr_off || !l->n_tasks || (mesh->n_entries > 0 && (!l->nbr_cell || !l->nbr_shift)))
        return HACC_ERR_INVALID;
    if (!l->tasks || !aligned16(l->tasks) || !l->task_order) return HACC_ERR_INVALID;
    // tasks above 64 particles: the gather kernels and the adjoints walk them in 64-particle
    // sub-chunks, the symmetric force kernel holds four i particles per lane
    if (l->split_T < 1 || l->split_T > 128) return HACC_ERR_INVALID;
    if (launch) {
        if (launch->warps_per_cta < 1 || launch->warps_per_cta > 8 || launch->ctas_per_sm < 1 ||
            launch->ctas_per_sm > 8 || launch->wait_cycles < 0)
            return HACC_ERR_INVALID;
    }
    if (ws_bytes < force_layout(mesh, nullptr).total) return HACC_ERR_CAPACITY;
    return HACC_OK;
}

// Arguments every pair kernel shares: the volumes, cells (or leaves), lists and tasks.
KArgs base_args(const hacc_mesh *mesh, const hacc_binned *binned, const hacc_lists *lists, const hacc_sr_params *p,
                uint32_t *status)
{
    KArgs a{};
    a.vols = mesh->vols;
    a.cell_start = binned->cell_start;
    a.nbr_off = lists->nbr_off;
    a.nbr_cell = lists->nbr_cell;
    a.nbr_shift = lists->nbr_shift;
    a.tasks = reinterpret_cast<const int4 *>(lists->tasks);
    a.order = lists->task_order;
    a.n_tasks = lists->n_tasks;
    a.origin = reinterpret_cast<const float4 *>(binned->cell_origin);
    a.pos = reinterpret_cast<const float4 *>(binned->sorted4);
    a.perm = binned->perm;
    a.mass_varies = binned->mass_varies;
    a.status = status;
    a.wait_limit = WAIT_LIMIT_CYCLES;
    a.N = mesh->N;
    a.n_cells = mesh->n_cells;
    a.n_entries = mesh->n_entries;
    a.task_cap = lists->task_cap;
    a.V = mesh->V;
    pair_consts(p, a.k);
    return a;
}

// The wait bound a launch asks for (0: the default).
long long wait_limit_of(const hacc_launch &L) { return L.wait_cycles > 0 ? (long long)L.wait_cycles : WAIT_LIMIT_CYCLES; }

}  // namespace
}  // namespace hacc

// Recursive coordinate bisection (RCB) fat-leaf tree and its leaf-shared
// interaction lists: the paper's own short-range data structure (Sec. III),
// built here as an alternative to the chaining mesh.  The leaves play the
// cells for the pair kernels (per-leaf origins instead of c w).
//
// Build, level-synchronous.  All groups still to be split at one depth are
// processed together.  Their particles are cut into chunks of CHUNK slots (a
// chunk never spans two groups).  Per chunk one warp reduces the integer box
// and the coordinate sums into the group's statistics (integer atomics: exact
// and order-free); a second pass counts the particles that go left; a global scan
// over the chunks turns the counts into stable destinations; the scatter then
// writes every particle to the next level's buffer, or straight to the final
// buffer when its half is a leaf.  Halves that still need splitting become
// the next level's groups, numbered by a scan (deterministic).  The host reads
// the number of groups left once per level.
//
// Walk.  One thread per leaf, depth first through its volume's tree, once per
// periodic image (27), skipping every node whose widened box is too far; the
// leaves come out in ascending id for each image (depth-first, left-first
// order is slot order).
#include <limits.h>
#include <math.h>

#include "hacc_common.cuh"

namespace hacc {
namespace {

constexpr int QBITS = HACC_RCB_QBITS;
constexpr int CHUNK = 256;        // slots per chunk; one warp per chunk
constexpr int IPT = CHUNK / 32;   // consecutive slots per lane in the scatter
constexpr int STACK = HACC_RCB_MAX_DEPTH + 2;
constexpr int32_t EMPTY_ROOT = INT_MIN;

struct GroupStat {
    int32_t lo[3];
    int32_t hi[3];
    unsigned long long sum[3];
    int32_t pad[4];
};
static_assert(sizeof(GroupStat) == 64, "GroupStat is 64 bytes");

// A group: slots [b, e), node id, depth.
__device__ __forceinline__ int4 make_group(int b, int e, int node, int depth) { return make_int4(b, e, node, depth); }

// floor(xw 2^21 / L), the quotient and product in float64, clamped to the grid.
__device__ __forceinline__ int32_t quant(float xw, float L)
{
    const double f = floor(__dmul_rn((double)xw, __ddiv_rn((double)(1 << QBITS), (double)L)));
    if (!(f >= 0.0)) return 0;
    if (f > (double)((1 << QBITS) - 1)) return (1 << QBITS) - 1;
    return (int32_t)f;
}

__device__ __forceinline__ float finite_or_zero(float v, bool &bad)
{
    if (isfinite(v)) return v;
    bad = true;
    return 0.0f;
}

struct Split {
    int axis;
    bool point;  // the box is a point: halve by position
    unsigned long long split;
};

// The splitting plane of a group: longest side (lowest axis on ties), floor of the mean.
__device__ __forceinline__ Split decide(const GroupStat &g, int cnt)
{
    Split s;
    s.axis = 0;
    for (int a = 1; a < 3; ++a)
        if (g.hi[a] - g.lo[a] > g.hi[s.axis] - g.lo[s.axis]) s.axis = a;
    s.point = g.hi[s.axis] == g.lo[s.axis];
    s.split = g.sum[s.axis] / (unsigned long long)cnt;
    return s;
}

__device__ __forceinline__ int coord(const int4 &q, int axis) { return axis == 0 ? q.x : (axis == 1 ? q.y : q.z); }

__device__ __forceinline__ bool goes_left(const Split &sp, const int4 &q, int rel, int cnt)
{
    return sp.point ? rel < cnt / 2 : (unsigned long long)coord(q, sp.axis) <= sp.split;
}

__device__ __forceinline__ bool is_leaf(int cnt, int depth, int leaf_max, int max_depth)
{
    return cnt <= leaf_max || depth >= max_depth;
}

// Group owning chunk c: the last s < S with chunk_base[s] <= c (every group has a chunk).
__device__ __forceinline__ int group_of_chunk(const int32_t *chunk_base, int S, int c)
{
    int lo = 0, hi = S - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (chunk_base[mid] <= c) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// build kernels
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(256)
k_rcb_init(const hacc_volume *__restrict__ vols, int V, const float *__restrict__ x, const float *__restrict__ y,
           const float *__restrict__ z, int64_t N, int leaf_max, int max_depth, int4 *__restrict__ qa,
           int4 *__restrict__ fin, int32_t *__restrict__ head, uint32_t *status)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
        const hacc_volume &vol = vols[find_volume_by_particle(vols, V, k)];
        bool bad = false;
        const float L = vol.L;
        const int4 q = make_int4(quant(wrap32(finite_or_zero(x[k], bad), L), L),
                                 quant(wrap32(finite_or_zero(y[k], bad), L), L),
                                 quant(wrap32(finite_or_zero(z[k], bad), L), L), (int)k);
        if (bad) atomicOr(status, HACC_STATUS_NONFINITE);
        const bool leaf_volume = is_leaf((int)(vol.p_end - vol.p_begin), 0, leaf_max, max_depth);
        if (leaf_volume) fin[k] = q; else qa[k] = q;
        head[k] = (leaf_volume && k == vol.p_begin) ? 1 : 0;
    }
}

// Roots, in volume order: empty, one leaf, or the first groups (node id = group index).
__global__ void k_rcb_roots(const hacc_volume *__restrict__ vols, int V, int leaf_max, int max_depth,
                            int4 *__restrict__ grp, int32_t *__restrict__ S0, int32_t *__restrict__ lvl_base,
                            int32_t *__restrict__ root)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    int s = 0;
    for (int v = 0; v < V; ++v) {
        const int b = (int)vols[v].p_begin, e = (int)vols[v].p_end;
        if (e == b) {
            root[v] = EMPTY_ROOT;
        } else if (is_leaf(e - b, 0, leaf_max, max_depth)) {
            root[v] = -1 - b;  // by first slot; turned into a leaf id at the end
        } else {
            grp[s] = make_group(b, e, s, 0);
            root[v] = s;
            ++s;
        }
    }
    *S0 = s;
    lvl_base[0] = 0;
}

__global__ void __launch_bounds__(256)
k_rcb_prep(const int4 *__restrict__ grp, const int32_t *__restrict__ S_in, int64_t Smax,
           GroupStat *__restrict__ stat, int32_t *__restrict__ nchunk)
{
    const int S = *S_in;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < Smax; s += (int64_t)gridDim.x * blockDim.x) {
        if (s >= S) {
            nchunk[s] = 0;
            continue;
        }
        const int4 g = grp[s];
        nchunk[s] = (g.y - g.x + CHUNK - 1) / CHUNK;
        GroupStat st;
        for (int a = 0; a < 3; ++a) {
            st.lo[a] = INT_MAX;
            st.hi[a] = -1;
            st.sum[a] = 0ull;
        }
        for (int a = 0; a < 4; ++a) st.pad[a] = 0;
        stat[s] = st;
    }
}

__device__ __forceinline__ int warp_min(int v)
{
    return __reduce_min_sync(0xffffffffu, v);
}
__device__ __forceinline__ int warp_max(int v)
{
    return __reduce_max_sync(0xffffffffu, v);
}
__device__ __forceinline__ unsigned long long warp_sum64(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Group of every chunk of the level (the last s < S with chunk_base[s] <= c).
__global__ void __launch_bounds__(256)
k_rcb_chunk_map(const int32_t *__restrict__ S_in, const int32_t *__restrict__ chunk_base, int64_t Smax,
                int32_t *__restrict__ chunk_group)
{
    const int S = *S_in;
    const int total = chunk_base[Smax];
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < total; c += gridDim.x * blockDim.x)
        chunk_group[c] = group_of_chunk(chunk_base, S, c);
}

// Per chunk (one warp): integer box and coordinate sums, merged into the group by atomics.
__global__ void __launch_bounds__(256)
k_rcb_reduce(const int4 *__restrict__ grp, const int32_t *__restrict__ chunk_base,
             const int32_t *__restrict__ chunk_group, int64_t Smax, const int4 *__restrict__ qa,
             GroupStat *__restrict__ stat)
{
    const int total = chunk_base[Smax];
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < total; c += warps) {
        const int s = chunk_group[c];
        const int4 g = grp[s];
        const int p0 = g.x + (c - chunk_base[s]) * CHUNK;
        const int p1 = min(g.y, p0 + CHUNK);
        int lo[3] = {INT_MAX, INT_MAX, INT_MAX}, hi[3] = {-1, -1, -1};
        unsigned long long sm[3] = {0ull, 0ull, 0ull};
        for (int p = p0 + lane; p < p1; p += 32) {
            const int4 q = qa[p];
            const int v[3] = {q.x, q.y, q.z};
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                lo[a] = min(lo[a], v[a]);
                hi[a] = max(hi[a], v[a]);
                sm[a] += (unsigned long long)v[a];
            }
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            lo[a] = warp_min(lo[a]);
            hi[a] = warp_max(hi[a]);
            sm[a] = warp_sum64(sm[a]);
        }
        if (lane < 3) {
            const int a = lane;
            atomicMin(&stat[s].lo[a], a == 0 ? lo[0] : (a == 1 ? lo[1] : lo[2]));
            atomicMax(&stat[s].hi[a], a == 0 ? hi[0] : (a == 1 ? hi[1] : hi[2]));
            atomicAdd(&stat[s].sum[a], a == 0 ? sm[0] : (a == 1 ? sm[1] : sm[2]));
        }
    }
}

// Per chunk (one warp): how many of its particles go left.
__global__ void __launch_bounds__(256)
k_rcb_count(const int4 *__restrict__ grp, const int32_t *__restrict__ chunk_base,
            const int32_t *__restrict__ chunk_group, int64_t Smax, const int4 *__restrict__ qa,
            const GroupStat *__restrict__ stat, int32_t *__restrict__ chunk_left)
{
    const int total = chunk_base[Smax];
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < total; c += warps) {
        const int s = chunk_group[c];
        const int4 g = grp[s];
        const int cnt = g.y - g.x;
        const Split sp = decide(stat[s], cnt);
        const int p0 = g.x + (c - chunk_base[s]) * CHUNK;
        const int p1 = min(g.y, p0 + CHUNK);
        int n = 0;
        for (int p = p0 + lane; p < p1; p += 32) n += goes_left(sp, qa[p], p - g.x, cnt) ? 1 : 0;
        n = __reduce_add_sync(0xffffffffu, n);
        if (lane == 0) chunk_left[c] = n;
    }
}

// Per chunk (one warp, IPT consecutive slots per lane): stable destinations;
// halves that are leaves go to the final buffer.
__global__ void __launch_bounds__(256)
k_rcb_scatter(const int4 *__restrict__ grp, const int32_t *__restrict__ chunk_base,
              const int32_t *__restrict__ chunk_group, const int32_t *__restrict__ chunk_loff, int64_t Smax,
              const int4 *__restrict__ qa, const GroupStat *__restrict__ stat, int leaf_max, int max_depth,
              int4 *__restrict__ qb, int4 *__restrict__ fin)
{
    const int total = chunk_base[Smax];
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c < total; c += warps) {
        const int s = chunk_group[c];
        const int4 g = grp[s];
        const int cnt = g.y - g.x;
        const Split sp = decide(stat[s], cnt);
        const int c0 = chunk_base[s], c1 = chunk_base[s + 1];
        const int nl = chunk_loff[c1] - chunk_loff[c0];
        const int lb = chunk_loff[c] - chunk_loff[c0];  // left particles of the group before this chunk
        const int p0 = g.x + (c - c0) * CHUNK;
        const int p1 = min(g.y, p0 + CHUNK);
        const bool leaf_l = is_leaf(nl, g.w + 1, leaf_max, max_depth);
        const bool leaf_r = is_leaf(cnt - nl, g.w + 1, leaf_max, max_depth);
        const int r0 = lane * IPT;  // this lane's slots p0 + r0 .. + IPT - 1
        int4 q[IPT];
        unsigned flags = 0;
        int n = 0;
#pragma unroll
        for (int j = 0; j < IPT; ++j) {
            const int p = p0 + r0 + j;
            if (p < p1) {
                q[j] = qa[p];
                if (goes_left(sp, q[j], p - g.x, cnt)) {
                    flags |= 1u << j;
                    ++n;
                }
            }
        }
        int incl = n;  // exclusive warp scan of the lanes' left counts: left slots of the chunk before r0
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        int left_before = incl - n;
        const int rb = (p0 - g.x) - lb;  // right particles of the group before this chunk
#pragma unroll
        for (int j = 0; j < IPT; ++j) {
            const int p = p0 + r0 + j;
            if (p >= p1) break;
            const int r = p - p0;  // slot within the chunk
            if (flags & (1u << j)) {
                const int dst = g.x + lb + left_before;
                if (leaf_l) fin[dst] = q[j]; else qb[dst] = q[j];
                ++left_before;
            } else {
                const int dst = g.x + nl + rb + (r - left_before);
                if (leaf_r) fin[dst] = q[j]; else qb[dst] = q[j];
            }
        }
    }
}

// Per group: node box, number of halves that are still groups.
__global__ void __launch_bounds__(256)
k_rcb_next(const int4 *__restrict__ grp, const int32_t *__restrict__ S_in, const int32_t *__restrict__ chunk_base,
           const int32_t *__restrict__ chunk_loff, int64_t Smax, const GroupStat *__restrict__ stat, int leaf_max,
           int max_depth, int64_t cap, int32_t *__restrict__ node_qbox, int32_t *__restrict__ kids, uint32_t *status)
{
    const int S = *S_in;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < Smax; s += (int64_t)gridDim.x * blockDim.x) {
        if (s >= S) {
            kids[s] = 0;
            continue;
        }
        const int4 g = grp[s];
        const int nl = chunk_loff[chunk_base[s + 1]] - chunk_loff[chunk_base[s]];
        const int cnt = g.y - g.x;
        kids[s] = (is_leaf(nl, g.w + 1, leaf_max, max_depth) ? 0 : 1) +
                  (is_leaf(cnt - nl, g.w + 1, leaf_max, max_depth) ? 0 : 1);
        if (g.z < cap) {
            const GroupStat st = stat[s];
            for (int a = 0; a < 3; ++a) {
                node_qbox[6 * (int64_t)g.z + a] = st.lo[a];
                node_qbox[6 * (int64_t)g.z + 3 + a] = st.hi[a];
            }
        } else {
            atomicOr(status, HACC_STATUS_CAPACITY);
        }
    }
}

// Per group: the next level's groups, the node's children, the leaf heads.
__global__ void __launch_bounds__(256)
k_rcb_link(const int4 *__restrict__ grp, const int32_t *__restrict__ S_in, const int32_t *__restrict__ chunk_base,
           const int32_t *__restrict__ chunk_loff, const int32_t *__restrict__ kid_off, int64_t Smax, int level,
           int leaf_max, int max_depth, int64_t cap, int4 *__restrict__ grp_next, int32_t *__restrict__ S_out,
           int32_t *__restrict__ lvl_base, int32_t *__restrict__ node_child, int32_t *__restrict__ head)
{
    const int S = *S_in;
    const int base_next = lvl_base[level] + S;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < S; s += (int64_t)gridDim.x * blockDim.x) {
        const int4 g = grp[s];
        const int nl = chunk_loff[chunk_base[s + 1]] - chunk_loff[chunk_base[s]];
        int slot = kid_off[s];
        int child[2];
        const int hb[2] = {g.x, g.x + nl}, he[2] = {g.x + nl, g.y};
        for (int h = 0; h < 2; ++h) {
            if (is_leaf(he[h] - hb[h], g.w + 1, leaf_max, max_depth)) {
                head[hb[h]] = 1;
                child[h] = -1 - hb[h];  // by first slot; turned into a leaf id at the end
            } else {
                child[h] = base_next + slot;
                grp_next[slot] = make_group(hb[h], he[h], base_next + slot, g.w + 1);
                ++slot;
            }
        }
        if (g.z < cap) {
            node_child[2 * (int64_t)g.z] = child[0];
            node_child[2 * (int64_t)g.z + 1] = child[1];
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        lvl_base[level + 1] = base_next;
        *S_out = kid_off[Smax];
    }
}

// Leaf starts from the head flags and their exclusive scan.
__global__ void __launch_bounds__(256)
k_rcb_leaf_starts(const int32_t *__restrict__ head, const int32_t *__restrict__ leaf_of_pos, int64_t N, int64_t cap,
                  int32_t *__restrict__ leaf_start, int32_t *__restrict__ n_leaves, const int32_t *__restrict__ lvl_base,
                  int levels, int32_t *__restrict__ n_nodes, uint32_t *status)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
        if (!head[k]) continue;
        const int l = leaf_of_pos[k];
        if (l < cap) leaf_start[l] = (int32_t)k;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        int64_t nl = leaf_of_pos[N];
        const int64_t nn = lvl_base[levels];
        if (nl > cap || nn > cap) atomicOr(status, HACC_STATUS_CAPACITY);
        if (nl > cap) nl = cap;
        *n_leaves = (int32_t)nl;
        *n_nodes = (int32_t)(nn < cap ? nn : cap);
        leaf_start[nl] = (int32_t)N;
    }
}

// One warp per leaf: box, origin, and the sorted records of its particles.
__global__ void __launch_bounds__(256)
k_rcb_leaf_fill(const hacc_volume *__restrict__ vols, int V, const float *__restrict__ x, const float *__restrict__ y,
                const float *__restrict__ z, const float *__restrict__ m, const int4 *__restrict__ fin,
                const int32_t *__restrict__ leaf_start, const int32_t *__restrict__ n_leaves,
                int32_t *__restrict__ leaf_qbox, float4 *__restrict__ leaf_origin, int32_t *__restrict__ perm,
                float4 *__restrict__ sorted4, int32_t *__restrict__ cell_of, uint32_t *mass_varies)
{
    MassCheck mc(m, mass_varies);
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int nl = *n_leaves;
    for (int64_t l = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); l < nl; l += warps) {
        const int b = leaf_start[l], e = leaf_start[l + 1];
        int lo[3] = {INT_MAX, INT_MAX, INT_MAX}, hi[3] = {-1, -1, -1};
        for (int k = b + lane; k < e; k += 32) {
            const int4 q = fin[k];
            lo[0] = min(lo[0], q.x); lo[1] = min(lo[1], q.y); lo[2] = min(lo[2], q.z);
            hi[0] = max(hi[0], q.x); hi[1] = max(hi[1], q.y); hi[2] = max(hi[2], q.z);
        }
        for (int a = 0; a < 3; ++a) {
            lo[a] = warp_min(lo[a]);
            hi[a] = warp_max(hi[a]);
        }
        const hacc_volume &vol = vols[find_volume_by_particle(vols, V, b)];
        const float L = vol.L;
        const double scale = __ddiv_rn((double)L, (double)(1 << QBITS));
        const float ox = __double2float_rn(__dmul_rn((double)lo[0], scale));
        const float oy = __double2float_rn(__dmul_rn((double)lo[1], scale));
        const float oz = __double2float_rn(__dmul_rn((double)lo[2], scale));
        if (lane < 6) leaf_qbox[6 * l + lane] = lane < 3 ? lo[lane] : hi[lane - 3];
        if (lane == 0) leaf_origin[l] = make_float4(ox, oy, oz, 0.0f);
        for (int k = b + lane; k < e; k += 32) {
            const int i = fin[k].w;
            bool bad = false;
            const float xw = wrap32(finite_or_zero(x[i], bad), L);
            const float yw = wrap32(finite_or_zero(y[i], bad), L);
            const float zw = wrap32(finite_or_zero(z[i], bad), L);
            perm[k] = i;
            const float mi = m[i];
            sorted4[k] = make_float4(__double2float_rn(__dsub_rn((double)xw, (double)ox)),
                                     __double2float_rn(__dsub_rn((double)yw, (double)oy)),
                                     __double2float_rn(__dsub_rn((double)zw, (double)oz)), mi);
            mc.check(mi);
            if (cell_of) cell_of[i] = (int32_t)l;
        }
    }
    mc.finish();
}

// Children and roots recorded by first slot become leaf ids.
__global__ void __launch_bounds__(256)
k_rcb_fix_children(const int32_t *__restrict__ leaf_of_pos, const int32_t *__restrict__ n_nodes, int V,
                   int32_t *__restrict__ node_child, int32_t *__restrict__ root)
{
    const int64_t nn = *n_nodes;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < 2 * nn + V;
         t += (int64_t)gridDim.x * blockDim.x) {
        int32_t *p = t < 2 * nn ? &node_child[t] : &root[t - 2 * nn];
        const int32_t c = *p;
        if (c < 0 && c != EMPTY_ROOT) *p = -1 - leaf_of_pos[-1 - c];
    }
}

// ---------------------------------------------------------------------------
// walk kernels
// ---------------------------------------------------------------------------

// Leaf test of the lists, exactly as the definition states it: boxes on the
// 2^21 grid widened by one step on every side, shifted by s L, sum of squared
// gaps in float64 (fixed order x, y, z) below rc^2.
__device__ __forceinline__ bool leaves_within_f64(const int32_t *qi, const int32_t *qj, double scale,
                                                  const double shL[3], double rc2)
{
    double d2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        const double ilo = __dmul_rn((double)(qi[a] - 1), scale), ihi = __dmul_rn((double)(qi[3 + a] + 2), scale);
        const double jlo = __dadd_rn(__dmul_rn((double)(qj[a] - 1), scale), shL[a]);
        const double jhi = __dadd_rn(__dmul_rn((double)(qj[3 + a] + 2), scale), shL[a]);
        double g = 0.0;
        const double t1 = __dsub_rn(jlo, ihi);
        if (t1 > g) g = t1;
        const double t2 = __dsub_rn(ilo, jhi);
        if (t2 > g) g = t2;
        d2 = __dadd_rn(d2, __dmul_rn(g, g));
    }
    return d2 < rc2;
}

// The same gaps counted in grid steps, exactly, in integers: one step is
// L / 2^21 and the image shift is s 2^21 steps.  The float64 sum of the
// definition differs from G steps^2 by far less than a step^2 near the
// cutoff (a few float64 roundings of values below 3 L), so G above
// (rc / step)^2 (1 + 1e-9) + 4 means the float64 test fails and G below
// (rc / step)^2 (1 - 1e-9) - 4 means it passes.
__device__ __forceinline__ long long gap2_steps(const int32_t *qi, const int32_t *qj, const long long shq[3])
{
    long long G = 0;
    for (int a = 0; a < 3; ++a) {
        const long long ilo = (long long)qi[a] - 1, ihi = (long long)qi[3 + a] + 2;
        const long long jlo = (long long)qj[a] - 1 + shq[a], jhi = (long long)qj[3 + a] + 2 + shq[a];
        long long g = 0;
        if (jlo - ihi > g) g = jlo - ihi;
        if (ilo - jhi > g) g = ilo - jhi;
        G += g * g;
    }
    return G;
}

// One thread per leaf: count (FILL = false) or write (FILL = true) its list.
template <bool FILL>
__global__ void __launch_bounds__(128)
k_rcb_walk(const hacc_volume *__restrict__ vols, int V, const int32_t *__restrict__ n_leaves,
           const int32_t *__restrict__ n_nodes, int64_t leaf_cap,
           const int32_t *__restrict__ leaf_start, const int32_t *__restrict__ leaf_qbox,
           const int32_t *__restrict__ node_qbox, const int32_t *__restrict__ node_child,
           const int32_t *__restrict__ root, int32_t *__restrict__ counts, unsigned long long *__restrict__ total,
           const int64_t *__restrict__ nbr_off, int64_t entry_cap, int32_t *__restrict__ nbr_leaf,
           int8_t *__restrict__ nbr_shift, uint32_t *status)
{
    const int nl = *n_leaves;
    const int nn = *n_nodes;
    unsigned long long mine = 0;
    for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < leaf_cap;
         l += (int64_t)gridDim.x * blockDim.x) {
        if (l >= nl) {
            if (!FILL) counts[l] = 0;
            continue;
        }
        const int v = find_volume_by_particle(vols, V, leaf_start[l]);
        const hacc_volume &vol = vols[v];
        const double Ld = (double)vol.L;
        const double scale = __ddiv_rn(Ld, (double)(1 << QBITS));
        const double rc2 = __dmul_rn((double)vol.rcut, (double)vol.rcut);
        const double Tq = rc2 / (scale * scale);  // the cutoff in steps^2 (margins below cover rounding)
        const double T_hi = Tq * (1.0 + 1e-9) + 4.0, T_lo = Tq * (1.0 - 1e-9) - 4.0;
        int32_t qi[6];
        for (int a = 0; a < 6; ++a) qi[a] = leaf_qbox[6 * l + a];
        const int32_t r = root[v];
        int64_t e = FILL ? nbr_off[l] : 0;
        int32_t n = 0;
        int32_t stack[STACK];
        for (int code = 0; code < 27; ++code) {
            const int sh[3] = {code % 3 - 1, (code / 3) % 3 - 1, code / 9 - 1};
            const double shL[3] = {(double)sh[0] * Ld, (double)sh[1] * Ld, (double)sh[2] * Ld};
            const long long shq[3] = {(long long)sh[0] << QBITS, (long long)sh[1] << QBITS,
                                      (long long)sh[2] << QBITS};
            int sp = 0;
            stack[sp++] = r;
            while (sp > 0) {
                const int32_t node = stack[--sp];
                if (node >= nn || node < -nl) {  // only a tree that ran out of capacity has these
                    atomicOr(status, HACC_STATUS_CAPACITY);
                    continue;
                }
                if (node >= 0) {
                    // an internal node is skipped only when the integer test proves every leaf below fails
                    if ((double)gap2_steps(qi, node_qbox + 6 * (int64_t)node, shq) > T_hi) continue;
                    if (sp + 2 > STACK) {  // deeper than any tree the build makes
                        atomicOr(status, HACC_STATUS_CAPACITY);
                        sp = 0;
                        break;
                    }
                    stack[sp++] = node_child[2 * (int64_t)node + 1];
                    stack[sp++] = node_child[2 * (int64_t)node];
                } else {
                    const int32_t j = -1 - node;
                    const int32_t *qj = leaf_qbox + 6 * (int64_t)j;
                    const double G = (double)gap2_steps(qi, qj, shq);
                    if (G > T_hi) continue;
                    if (!(G < T_lo) && !leaves_within_f64(qi, qj, scale, shL, rc2)) continue;
                    if (FILL) {
                        if (e < entry_cap) {
                            nbr_leaf[e] = j;
                            nbr_shift[e] = (int8_t)code;
                        }
                        ++e;
                    } else {
                        ++n;
                    }
                }
            }
        }
        if (!FILL) {
            counts[l] = n;
            mine += (unsigned long long)n;
        }
    }
    if (!FILL) {
        mine = warp_sum64(mine);
        if ((threadIdx.x & 31) == 0 && mine) atomicAdd(total, mine);
    }
}

__global__ void __launch_bounds__(256)
k_rcb_offsets(const int32_t *__restrict__ offs, int64_t leaf_cap, int64_t *__restrict__ nbr_off)
{
    for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l <= leaf_cap;
         l += (int64_t)gridDim.x * blockDim.x)
        nbr_off[l] = offs[l];
}

__global__ void k_rcb_entries_check(const unsigned long long *__restrict__ total, int64_t entry_cap,
                                    int64_t *__restrict__ n_entries, int32_t *__restrict__ fits, uint32_t *status)
{
    const unsigned long long t = *total;
    *n_entries = (int64_t)t;
    const bool ok = t <= (unsigned long long)entry_cap && t <= (unsigned long long)INT_MAX;
    *fits = ok ? 1 : 0;
    if (!ok && status) atomicOr(status, HACC_STATUS_CAPACITY);
}

// Tasks: each leaf cut into chunks of at most T particles.
__global__ void __launch_bounds__(256)
k_rcb_task_counts(const int32_t *__restrict__ leaf_start, const int32_t *__restrict__ n_leaves, int64_t leaf_cap,
                  int T, int32_t *__restrict__ nt)
{
    const int nl = *n_leaves;
    for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < leaf_cap;
         l += (int64_t)gridDim.x * blockDim.x)
        nt[l] = l < nl ? (leaf_start[l + 1] - leaf_start[l] + T - 1) / T : 0;
}

__global__ void __launch_bounds__(256)
k_rcb_task_fill(const hacc_volume *__restrict__ vols, int V, const int32_t *__restrict__ leaf_start,
                const int32_t *__restrict__ n_leaves, int T, const int32_t *__restrict__ task_off, int64_t cap,
                int4 *__restrict__ tasks)
{
    const int nl = *n_leaves;
    for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < nl; l += (int64_t)gridDim.x * blockDim.x) {
        const int b = leaf_start[l], e = leaf_start[l + 1];
        const int v = find_volume_by_particle(vols, V, b);
        int64_t t = task_off[l];
        for (int i = b; i < e && t < cap; i += T, ++t) tasks[t] = make_int4((int)l, i, min(i + T, e), v);
    }
}

// Candidate ordered pairs: sum over leaves of count(l) * sum_list count(l').
__global__ void __launch_bounds__(256)
k_rcb_pair_count(const int32_t *__restrict__ leaf_start, const int32_t *__restrict__ n_leaves,
                 const int64_t *__restrict__ nbr_off, const int32_t *__restrict__ nbr_leaf,
                 const int32_t *__restrict__ fits, unsigned long long *__restrict__ acc_total)
{
    const int nl = *fits ? *n_leaves : 0;
    unsigned long long acc = 0;
    for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < nl; l += (int64_t)gridDim.x * blockDim.x) {
        const int64_t ni = leaf_start[l + 1] - leaf_start[l];
        int64_t nj = 0;
        for (int64_t e = nbr_off[l]; e < nbr_off[l + 1]; ++e) {
            const int j = nbr_leaf[e];
            nj += leaf_start[j + 1] - leaf_start[j];
        }
        acc += (unsigned long long)(ni * nj);
    }
    acc = warp_sum64(acc);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(acc_total, acc);
}

__global__ void k_rcb_lists_finish(const int32_t *__restrict__ task_off, int64_t leaf_cap, int64_t cap, int64_t N,
                                   const unsigned long long *__restrict__ pairs, int32_t *__restrict__ n_tasks,
                                   int64_t *__restrict__ n_pairs, uint32_t *status)
{
    int64_t t = task_off[leaf_cap];
    if (t > cap) {
        atomicOr(status, HACC_STATUS_CAPACITY);
        t = cap;
    }
    *n_tasks = (int32_t)t;
    if (n_pairs) *n_pairs = (int64_t)*pairs - N;  // each particle meets itself once, in its own leaf
}

// Heaviest-first cost class of each task slot (as for the chaining mesh).
__global__ void __launch_bounds__(256)
k_rcb_task_keys(const int4 *__restrict__ tasks, const int32_t *__restrict__ n_tasks, int64_t cap,
                const int32_t *__restrict__ leaf_start, const int64_t *__restrict__ nbr_off,
                const int32_t *__restrict__ nbr_leaf, const int32_t *__restrict__ fits, int32_t *__restrict__ keys)
{
    const int64_t nt = *n_tasks;
    const bool lists_ok = *fits != 0;  // entries past the capacity were not written
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < cap; t += (int64_t)gridDim.x * blockDim.x) {
        if (t >= nt) {
            keys[t] = 255;
            continue;
        }
        const int4 tk = tasks[t];
        int64_t nj = 0;
        for (int64_t e = nbr_off[tk.x]; lists_ok && e < nbr_off[tk.x + 1]; ++e) {
            const int j = nbr_leaf[e];
            nj += leaf_start[j + 1] - leaf_start[j];
        }
        const uint64_t cost = (uint64_t)(tk.z - tk.y) * (uint64_t)(nj > 0 ? nj : 1);
        keys[t] = 63 - (63 - __clzll((long long)cost));
    }
}

// ---------------------------------------------------------------------------
// workspaces
// ---------------------------------------------------------------------------

struct Carver {
    char *p;
    size_t off = 0;
    template <class T>
    T *take(size_t count)
    {
        T *q = p ? reinterpret_cast<T *>(p + off) : nullptr;
        off += round_up(count * sizeof(T), 256);
        return q;
    }
};

struct BuildWs {
    int4 *qa, *qb, *fin, *grp0, *grp1;
    int32_t *head, *leaf_of_pos, *nchunk, *chunk_base, *kids, *kid_off, *chunk_left, *chunk_loff, *chunk_group, *S,
        *lvl_base;
    GroupStat *stat;
    char *scan_ws;
    int64_t Smax, Cmax;
    size_t total;
};

BuildWs build_layout(int64_t N, int leaf_max, void *ws)
{
    BuildWs B{};
    B.Smax = N / ((int64_t)leaf_max + 1) + 1;
    B.Cmax = (N + CHUNK - 1) / CHUNK + B.Smax;
    Carver c{reinterpret_cast<char *>(ws)};
    const size_t n1 = (size_t)(N > 0 ? N : 1);
    B.qa = c.take<int4>(n1);
    B.qb = c.take<int4>(n1);
    B.fin = c.take<int4>(n1);
    B.head = c.take<int32_t>(n1 + 1);
    B.leaf_of_pos = c.take<int32_t>(n1 + 1);
    B.grp0 = c.take<int4>(B.Smax);
    B.grp1 = c.take<int4>(B.Smax);
    B.stat = c.take<GroupStat>(B.Smax);
    B.nchunk = c.take<int32_t>(B.Smax);
    B.chunk_base = c.take<int32_t>(B.Smax + 1);
    B.kids = c.take<int32_t>(B.Smax);
    B.kid_off = c.take<int32_t>(B.Smax + 1);
    B.chunk_left = c.take<int32_t>(B.Cmax);
    B.chunk_loff = c.take<int32_t>(B.Cmax + 1);
    B.chunk_group = c.take<int32_t>(B.Cmax);
    B.S = c.take<int32_t>(2);
    B.lvl_base = c.take<int32_t>(HACC_RCB_MAX_DEPTH + 2);
    int64_t ns = (int64_t)n1;
    if (B.Cmax > ns) ns = B.Cmax;
    if (B.Smax > ns) ns = B.Smax;
    B.scan_ws = c.take<char>(scan_workspace_bytes(ns));
    B.total = c.off;
    return B;
}

struct WalkWs {
    int32_t *counts, *offs, *nt, *task_off, *keys, *fits;
    unsigned long long *total, *pairs;
    char *scan_ws, *sort_ws;
    size_t total_bytes;
};

WalkWs walk_layout(int64_t leaf_cap, int64_t task_cap, void *ws)
{
    WalkWs W{};
    Carver c{reinterpret_cast<char *>(ws)};
    const size_t lc = (size_t)(leaf_cap > 0 ? leaf_cap : 1);
    W.counts = c.take<int32_t>(lc);
    W.offs = c.take<int32_t>(lc + 1);
    W.nt = c.take<int32_t>(lc);
    W.task_off = c.take<int32_t>(lc + 1);
    W.keys = c.take<int32_t>((size_t)(task_cap > 0 ? task_cap : 1));
    W.fits = c.take<int32_t>(1);
    W.total = c.take<unsigned long long>(1);
    W.pairs = c.take<unsigned long long>(1);
    W.scan_ws = c.take<char>(scan_workspace_bytes((int64_t)lc));
    W.sort_ws = c.take<char>(sort_workspace_bytes(task_cap > 0 ? task_cap : 1));
    W.total_bytes = c.off;
    return W;
}

int grid_for(int64_t n, int per_sm)
{
    int64_t g = (n + 255) / 256;
    const int64_t cap = (int64_t)num_sms() * per_sm;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

bool tree_ok(const hacc_tree *t)
{
    return t && t->leaf_max >= 1 && t->max_depth >= 0 && t->max_depth <= HACC_RCB_MAX_DEPTH && t->leaf_cap >= 1 &&
           t->n_leaves && t->n_nodes && t->leaf_start && t->leaf_qbox && t->leaf_origin && t->node_qbox &&
           t->node_child && t->root && aligned16(t->leaf_origin);
}

}  // namespace
}  // namespace hacc

using namespace hacc;

extern "C" size_t hacc_rcb_build_workspace_size(const hacc_mesh *mesh, int32_t leaf_max)
{
    if (!mesh || leaf_max < 1) return 0;
    return build_layout(mesh->N, leaf_max, nullptr).total;
}

extern "C" int hacc_rcb_build(const hacc_mesh *mesh, const float *x, const float *y, const float *z, const float *m,
                              const hacc_tree *tree, const hacc_binned *out, void *ws, size_t ws_bytes,
                              uint32_t *status, void *stream)
{
    if (!mesh || !mesh->vols || mesh->V < 1 || !tree_ok(tree) || !out || !status || !ws || !aligned16(ws))
        return HACC_ERR_INVALID;
    const int64_t N = mesh->N;
    if (N > 0 && (!x || !y || !z || !m || !out->perm || !out->sorted4 || !aligned16(out->sorted4)))
        return HACC_ERR_INVALID;
    if (N >= INT_MAX) return HACC_ERR_INVALID;
    BuildWs B = build_layout(N, tree->leaf_max, ws);
    if (ws_bytes < B.total) return HACC_ERR_CAPACITY;
    cudaStream_t st = as_stream(stream);
    const int V = mesh->V;
    const int lm = tree->leaf_max, md = tree->max_depth;
    const int64_t cap = tree->leaf_cap;

    if (out->mass_varies) HACC_CUDA_TRY(cudaMemsetAsync(out->mass_varies, 0, sizeof(uint32_t), st));
    if (N > 0) {
        // every final slot is written by exactly one scatter; cleared first so that no
        // index read from it can leave [0, N) whatever happens
        HACC_CUDA_TRY(cudaMemsetAsync(B.fin, 0, (size_t)N * sizeof(int4), st));
        k_rcb_init<<<grid_for(N, 16), 256, 0, st>>>(mesh->vols, V, x, y, z, N, lm, md, B.qa, B.fin, B.head, status);
        HACC_LAUNCH_CHECK();
    }
    k_rcb_roots<<<1, 32, 0, st>>>(mesh->vols, V, lm, md, B.grp0, &B.S[0], B.lvl_base, tree->root);
    HACC_LAUNCH_CHECK();

    int4 *qa = B.qa, *qb = B.qb, *grp = B.grp0, *grp_next = B.grp1;
    int32_t *S_in = &B.S[0], *S_out = &B.S[1];
    const int gs = grid_for(B.Smax, 16);
    const int gc = num_sms() * 8;  // chunk kernels (a warp per chunk): persistent over the level's chunks
    int level = 0;
    for (;; ++level) {
        int32_t h_S = 0;
        HACC_CUDA_TRY(cudaMemcpyAsync(&h_S, S_in, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        HACC_CUDA_TRY(cudaStreamSynchronize(st));
        if (h_S == 0 || level > HACC_RCB_MAX_DEPTH) break;
        k_rcb_prep<<<gs, 256, 0, st>>>(grp, S_in, B.Smax, B.stat, B.nchunk);
        HACC_LAUNCH_CHECK();
        int rc = scan_exclusive_i32(B.nchunk, B.chunk_base, B.Smax, B.scan_ws, st);
        if (rc) return rc;
        HACC_CUDA_TRY(cudaMemsetAsync(B.chunk_left, 0, (size_t)B.Cmax * sizeof(int32_t), st));
        k_rcb_chunk_map<<<grid_for(B.Cmax, 16), 256, 0, st>>>(S_in, B.chunk_base, B.Smax, B.chunk_group);
        HACC_LAUNCH_CHECK();
        k_rcb_reduce<<<gc, 256, 0, st>>>(grp, B.chunk_base, B.chunk_group, B.Smax, qa, B.stat);
        HACC_LAUNCH_CHECK();
        k_rcb_count<<<gc, 256, 0, st>>>(grp, B.chunk_base, B.chunk_group, B.Smax, qa, B.stat, B.chunk_left);
        HACC_LAUNCH_CHECK();
        rc = scan_exclusive_i32(B.chunk_left, B.chunk_loff, B.Cmax, B.scan_ws, st);
        if (rc) return rc;
        k_rcb_scatter<<<gc, 256, 0, st>>>(grp, B.chunk_base, B.chunk_group, B.chunk_loff, B.Smax, qa, B.stat, lm,
                                          md, qb, B.fin);
        HACC_LAUNCH_CHECK();
        k_rcb_next<<<gs, 256, 0, st>>>(grp, S_in, B.chunk_base, B.chunk_loff, B.Smax, B.stat, lm, md, cap,
                                       tree->node_qbox, B.kids, status);
        HACC_LAUNCH_CHECK();
        rc = scan_exclusive_i32(B.kids, B.kid_off, B.Smax, B.scan_ws, st);
        if (rc) return rc;
        k_rcb_link<<<gs, 256, 0, st>>>(grp, S_in, B.chunk_base, B.chunk_loff, B.kid_off, B.Smax, level, lm, md, cap,
                                       grp_next, S_out, B.lvl_base, tree->node_child, B.head);
        HACC_LAUNCH_CHECK();
        int4 *t4 = qa; qa = qb; qb = t4;
        t4 = grp; grp = grp_next; grp_next = t4;
        int32_t *ts = S_in; S_in = S_out; S_out = ts;
    }

    if (N > 0) {
        int rc = scan_exclusive_i32(B.head, B.leaf_of_pos, N, B.scan_ws, st);
        if (rc) return rc;
    } else {
        HACC_CUDA_TRY(cudaMemsetAsync(B.leaf_of_pos, 0, sizeof(int32_t), st));
    }
    k_rcb_leaf_starts<<<grid_for(N, 16), 256, 0, st>>>(B.head, B.leaf_of_pos, N, cap, tree->leaf_start,
                                                       tree->n_leaves, B.lvl_base, level, tree->n_nodes, status);
    HACC_LAUNCH_CHECK();
    if (N > 0) {
        k_rcb_leaf_fill<<<grid_for(N, 16), 256, 0, st>>>(mesh->vols, V, x, y, z, m, B.fin, tree->leaf_start,
                                                         tree->n_leaves, tree->leaf_qbox,
                                                         reinterpret_cast<float4 *>(tree->leaf_origin), out->perm,
                                                         reinterpret_cast<float4 *>(out->sorted4), out->cell_of,
                                                         out->mass_varies);
        HACC_LAUNCH_CHECK();
    }
    k_rcb_fix_children<<<grid_for(2 * (N / 2 + 1) + V, 16), 256, 0, st>>>(B.leaf_of_pos, tree->n_nodes, V,
                                                                          tree->node_child, tree->root);
    HACC_LAUNCH_CHECK();
    return HACC_OK;
}

extern "C" size_t hacc_rcb_lists_workspace_size(const hacc_mesh *mesh, int64_t leaf_cap, int64_t task_cap)
{
    if (!mesh || leaf_cap < 1 || task_cap < 0) return 0;
    return walk_layout(leaf_cap, task_cap, nullptr).total_bytes;
}

extern "C" int hacc_rcb_lists(const hacc_mesh *mesh, const hacc_tree *tree, const hacc_lists *lists,
                              int64_t entry_cap, int64_t *n_entries, void *ws, size_t ws_bytes, uint32_t *status,
                              void *stream)
{
    if (!mesh || !mesh->vols || mesh->V < 1 || !tree_ok(tree) || !lists || !n_entries || !status || !ws)
        return HACC_ERR_INVALID;
    if (!lists->nbr_off || entry_cap < 0) return HACC_ERR_INVALID;
    const bool fill = lists->nbr_cell != nullptr;
    if (fill) {
        if (!lists->nbr_shift || !lists->n_tasks || lists->split_T < 1 || lists->task_cap < 1 || !lists->tasks ||
            !aligned16(lists->tasks) || !lists->task_order)
            return HACC_ERR_INVALID;
    }
    const int64_t lc = tree->leaf_cap;
    WalkWs W = walk_layout(lc, fill ? lists->task_cap : 0, ws);
    if (ws_bytes < W.total_bytes) return HACC_ERR_CAPACITY;
    cudaStream_t st = as_stream(stream);
    const int V = mesh->V;
    const int gw = grid_for(lc, 64) * 2;  // 128-thread CTAs

    HACC_CUDA_TRY(cudaMemsetAsync(W.total, 0, sizeof(unsigned long long), st));
    k_rcb_walk<false><<<gw, 128, 0, st>>>(mesh->vols, V, tree->n_leaves, tree->n_nodes, lc, tree->leaf_start, tree->leaf_qbox,
                                          tree->node_qbox, tree->node_child, tree->root, W.counts, W.total, nullptr,
                                          0, nullptr, nullptr, status);
    HACC_LAUNCH_CHECK();
    int rc = scan_exclusive_i32(W.counts, W.offs, lc, W.scan_ws, st);
    if (rc) return rc;
    k_rcb_offsets<<<grid_for(lc + 1, 16), 256, 0, st>>>(W.offs, lc, lists->nbr_off);
    HACC_LAUNCH_CHECK();
    k_rcb_entries_check<<<1, 1, 0, st>>>(W.total, fill ? entry_cap : INT64_MAX, n_entries, W.fits,
                                         fill ? status : nullptr);
    HACC_LAUNCH_CHECK();
    if (!fill) return HACC_OK;

    // entries are written only where they fit (the walk checks each slot against entry_cap)
    k_rcb_walk<true><<<gw, 128, 0, st>>>(mesh->vols, V, tree->n_leaves, tree->n_nodes, lc, tree->leaf_start, tree->leaf_qbox,
                                         tree->node_qbox, tree->node_child, tree->root, nullptr, nullptr,
                                         lists->nbr_off, entry_cap, lists->nbr_cell, lists->nbr_shift, status);
    HACC_LAUNCH_CHECK();
    const int T = lists->split_T;
    k_rcb_task_counts<<<grid_for(lc, 16), 256, 0, st>>>(tree->leaf_start, tree->n_leaves, lc, T, W.nt);
    HACC_LAUNCH_CHECK();
    rc = scan_exclusive_i32(W.nt, W.task_off, lc, W.scan_ws, st);
    if (rc) return rc;
    k_rcb_task_fill<<<grid_for(lc, 16), 256, 0, st>>>(mesh->vols, V, tree->leaf_start, tree->n_leaves, T, W.task_off,
                                                      lists->task_cap, reinterpret_cast<int4 *>(lists->tasks));
    HACC_LAUNCH_CHECK();
    HACC_CUDA_TRY(cudaMemsetAsync(W.pairs, 0, sizeof(unsigned long long), st));
    k_rcb_pair_count<<<grid_for(lc, 16), 256, 0, st>>>(tree->leaf_start, tree->n_leaves, lists->nbr_off,
                                                       lists->nbr_cell, W.fits, W.pairs);
    HACC_LAUNCH_CHECK();
    k_rcb_lists_finish<<<1, 1, 0, st>>>(W.task_off, lc, lists->task_cap, mesh->N, W.pairs, lists->n_tasks,
                                        lists->n_pairs, status);
    HACC_LAUNCH_CHECK();
    k_rcb_task_keys<<<grid_for(lists->task_cap, 16), 256, 0, st>>>(
        reinterpret_cast<const int4 *>(lists->tasks), lists->n_tasks, lists->task_cap, tree->leaf_start,
        lists->nbr_off, lists->nbr_cell, W.fits, W.keys);
    HACC_LAUNCH_CHECK();
    return sort_index_stable(W.keys, lists->task_cap, 8, lists->task_order, W.sort_ws, st);
}

/*
 * hacc_sr.h -- C ABI of the GB300 short-range particle-particle force path.
 *
 * The method is the short-range half of HACC's force split (Habib et al.,
 * "The Universe at Extreme Scale: Multi-Petaflop Sky Simulation on the BG/Q",
 * SC'12; arXiv:1211.4864):
 *
 *   a_i = sum_{j != i, s_ij < r_c^2} m_j f_SR(s_ij) d_ij,
 *   f_SR(s) = (s + eps)^(-3/2) - poly[5](s),      s = d.d      (Eq. 7)
 *
 * where d_ij = x_j - x_i is the minimum periodic image, poly[5] is the
 * fifth-order fit of the filtered grid force (Sec. II), eps the short-distance
 * cutoff (softening, added to s) and r_c the matching radius of the force
 * split (3 grid cells, Sec. II).  The paper evaluates it with an RCB tree and
 * leaf-shared neighbour lists on the BG/Q (Sec. III); this library bins the
 * particles into a periodic chaining mesh (cell width >= the mesh's minimum
 * width), builds per-cell neighbour-cell lists, evaluates the pair force on the
 * GPU, and applies the kick of the split-operator step (Eq. 6).
 *
 * Conventions for every call
 * --------------------------
 *  * All array pointers are DEVICE pointers owned by the caller, unless the
 *    comment says "host".  The library allocates no device memory: scratch
 *    space is passed in as `ws` of at least the size that the matching
 *    *_workspace_size query returns.  Float4 arrays (`sorted4`) and `ws` must
 *    be 16-byte aligned.
 *  * `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Calls only enqueue work on it; nothing synchronises the host, so a
 *    sequence of calls can be captured in a CUDA graph.
 *  * Return value: HACC_OK, or a negative code for an error found on the host
 *    (bad argument, CUDA launch error).  Errors that only the device can see
 *    (a full task buffer, a wait that ran out, a non-finite coordinate) are
 *    OR-ed as HACC_STATUS_* bits into the caller's device word `status`; read
 *    it after the stream has finished.  No C++ exception crosses the ABI.
 *  * Several volumes: every call works on V >= 1 independent periodic boxes
 *    whose particles are concatenated; a one-box problem is V = 1.
 *  * Particle counts are below 2^31.
 */
#ifndef HACC_SR_H
#define HACC_SR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HACC_OK 0
#define HACC_ERR_INVALID (-1)  /* bad argument (checked on the host) */
#define HACC_ERR_CAPACITY (-2) /* a buffer or workspace is too small */
#define HACC_ERR_CUDA (-3)     /* a CUDA call failed */
#define HACC_ERR_TIMEOUT (-4)  /* reserved for a host-side wait that ran out */

/* bits of the device status word */
#define HACC_STATUS_CAPACITY 1u /* task buffer too small: some tasks were dropped */
#define HACC_STATUS_TIMEOUT 2u  /* a bounded device wait gave up; results invalid */
#define HACC_STATUS_NONFINITE 4u /* a position was NaN or infinite (binned to 0) */
#define HACC_STATUS_SKIN 8u      /* a drifted offset left its cell widened by skin/2: re-bin */
#define HACC_STATUS_BOUNDS 16u   /* debug build only (libhacc_sr_debug.so, compiled with
                                    HACC_DEBUG_BOUNDS): an index read from the lists, tasks or
                                    binning was out of range; the work it led to was skipped */

/* One periodic volume of the chaining mesh (64 bytes).  Filled on the host by
 * hacc_mesh_plan, then copied by the caller to device memory. */
typedef struct hacc_volume {
    int64_t p_begin;    /* first particle of this volume */
    int64_t p_end;      /* one past its last particle */
    int64_t cell_base;  /* global id of its first cell */
    int64_t entry_base; /* index of its first neighbour-list entry */
    int32_t n;          /* cells per side: floor(L / cell_min) */
    int32_t R;          /* stencil reach in cells: ceil(r_c / w) */
    int32_t S;          /* neighbour-list entries per cell */
    float L;            /* box side (grid units) */
    float w;            /* cell width, float32 L / n */
    float inv_w;        /* float32 n / L, used to find a particle's cell */
    float rcut;         /* cutoff the lists were planned for */
    int32_t pad;
} hacc_volume;

/* Mesh of V volumes as the device calls see it. */
typedef struct hacc_mesh {
    const hacc_volume *vols; /* device [V] */
    int32_t V;
    int32_t pad;
    int64_t N;         /* particles over all volumes (= vols[V-1].p_end) */
    int64_t n_cells;   /* cells over all volumes */
    int64_t n_entries; /* neighbour-list entries over all volumes */
} hacc_mesh;

/* Output of hacc_bin (chaining-mesh cells) or of hacc_rcb_build (tree
 * leaves, which then play the cells: cell_start = the tree's leaf_start,
 * cell_origin = its leaf_origin). */
typedef struct hacc_binned {
    int32_t *cell_of;    /* [N] global cell (leaf) of particle i (input order); may be NULL for the tree */
    int32_t *cell_start; /* [n_cells + 1] first sorted slot of each cell */
    int32_t *perm;       /* [N] input index of the particle in sorted slot k */
    float *sorted4;      /* [4 N] per sorted slot (ox, oy, oz, m), o = cell-relative offset */
    float *cell_origin;  /* [4 n_cells] (x, y, z, 0) origin the offsets of each cell are taken from,
                            or NULL for the chaining mesh (the offsets of cell (cx, cy, cz) are taken
                            from its centre, float32 (c + 1/2) w per axis) */
    uint32_t *mass_varies; /* device word or NULL.  hacc_bin, hacc_bin_noalloc and hacc_rcb_build set
                            it to 0 when every mass is bitwise equal to the first particle's (N = 0
                            included) and to 1 otherwise.  When it reads 0, the force calls
                            (hacc_sr_force, hacc_sr_force_symmetric) and the adjoint calls take
                            their equal-mass path: the pair sums hold f d (adjoint without gm:
                            W = sum f (lam_j - lam_i) + 2 f' (d.(lam_j - lam_i)) d; with gm:
                            V = sum f, X = sum 2 f' (d.(lam_j - lam_i)) d) and each particle's total is
                            scaled once by its own mass, the common m (sum_j m_j f d =
                            m sum_j f d), which saves per-pair mass products; the results agree
                            with the general path to float32 rounding.  NULL: the general path,
                            always. */
} hacc_binned;

/* Output of hacc_build_lists. */
typedef struct hacc_lists {
    int64_t *nbr_off;  /* [n_cells + 1] first entry of each cell's neighbour list */
    int32_t *nbr_cell; /* [n_entries] global id of the neighbour cell */
    int8_t *nbr_shift; /* [n_entries] periodic image: (sz+1)*9 + (sy+1)*3 + (sx+1) */
    int32_t *tasks;    /* [4 task_cap] per task: cell, first slot, end slot, volume */
    int32_t *n_tasks;  /* device scalar: number of tasks written */
    int64_t *n_pairs;  /* device scalar: candidate ordered pairs (j != i) the force visits */
    int32_t *task_order; /* [task_cap] the order the pair kernels take tasks in: by descending
                            cost class (particles x list length, power-of-two classes), stable */
    int64_t task_cap;  /* capacity of `tasks`, in tasks */
    int32_t split_T;   /* a task holds at most split_T particles of one cell; the pair calls take
                          1..128 (the symmetric force kernel runs a task of at most 16 particles
                          on two half-warps, then one, two or four i particles per lane; the
                          other pair kernels walk a task in 64-particle sub-chunks) */
    int32_t pad;
} hacc_lists;

/* Force-law parameters (host struct). */
typedef struct hacc_sr_params {
    float eps;  /* softening added to s (grid units^2), > 0 */
    float rcut; /* cutoff radius r_c (grid units); pairs with s < r_c^2 interact */
    float c[6]; /* poly[5] coefficients, poly(s) = sum_k c[k] s^k */
} hacc_sr_params;

/* Launch shape of the pair kernels (host struct; NULL = built-in default).
 * The autotuner picks these per workload. */
typedef struct hacc_launch {
    int32_t warps_per_cta; /* 1..8 */
    int32_t ctas_per_sm;   /* resident CTAs per SM of the persistent grid, 1..8 */
    int32_t jtile;         /* j particles per staged tile: 32, 64, 128 or 256 */
    int32_t stages;        /* staged tiles in flight per warp: 2..4 */
    int64_t wait_cycles;   /* bound of each wait for a staged tile, in SM clock cycles (clock64),
                              checked before every poll of the tile's mbarrier; 0 = the default
                              2e9 (about 1 s at 2 GHz), negative is invalid.  A warp whose wait runs
                              out sets HACC_STATUS_TIMEOUT, lets the copies it has in flight land
                              (waiting at most the default bound), and stops taking tasks; the
                              call's results are then invalid.  A bound of 1 makes every wait give
                              up at once although its copies complete: the failure path can be
                              exercised without a hang. */
} hacc_launch;

/* Library version and build target, e.g. "hacc_sr 1 sm_103a". Host. */
const char *hacc_version(void);

/* Reads the device status word `status` into the host word *value once the
 * work enqueued on `stream` so far has finished (synchronises `stream`).
 * HACC_ERR_CUDA if the copy or the wait fails (a fault of earlier work shows
 * here). */
int hacc_get_status(const uint32_t *status, uint32_t *value, void *stream);

/* Number of kernels this library has launched in this process so far (host;
 * a tracing aid: the difference across a region counts its launches). */
uint64_t hacc_kernel_launches(void);

/* Plans the chaining mesh of V volumes (host only, no device work).
 *   L[V]         host: box side of each volume (grid units), > 0
 *   vol_off[V+1] host: particle ranges, vol_off[0] = 0, non-decreasing
 *   cell_min     minimum cell width (normally r_c); n = floor(L / cell_min) >= 3
 *   rcut         cutoff; requires L >= 2 r_c and n >= 2 R + 1 (unique image)
 *   table[V]     host out: the volumes; copy it to the device for the calls
 *   out_mesh     host out: totals (its `vols` is left NULL for the caller)
 * The chaining mesh stands in for the paper's RCB tree (Sec. III).
 * Returns HACC_ERR_INVALID on any violated requirement. */
int hacc_mesh_plan(int32_t V, const float *L, const int64_t *vol_off, float cell_min, float rcut,
                   hacc_volume *table, hacc_mesh *out_mesh);

/* Bytes of scratch that hacc_bin needs. */
size_t hacc_bin_workspace_size(const hacc_mesh *mesh);

/* Bins the particles into the chaining mesh: the analogue of the paper's
 * three-phase structure-of-arrays partition (Sec. III), done as a stable
 * counting sort.  For particle i of volume v, per axis: xw = x - L floor(x/L)
 * (one correction step keeps xw in [0, L)), cell c = min(n-1, floor(xw inv_w)),
 * offset from the cell centre o = xw - fl32((c + 1/2) w) (|o| <= w/2), each a
 * single float32 round-to-nearest operation.
 * Optional displacements dx, dy, dz (all three or none, [N]): the position is
 * then x + d, formed, wrapped and offset in float64 (same steps, each one
 * float64 round-to-nearest operation, the cell from floor(xw inv_w) in
 * float64) and only the offset o = xw - fl32((c + 1/2) w) is rounded to float32; a
 * trajectory kept as a fixed reference plus a small drift displacement so
 * keeps its float64 position to float32 precision of a cell-relative offset.
 * Within a cell the sorted order is ascending input index (bit-exact and
 * deterministic).  x, y, z, m: [N] input order.  Writes every array of `out`
 * (out->mass_varies if not NULL).  N and n_cells below 2^31, else
 * HACC_ERR_INVALID.
 * A non-finite coordinate sets HACC_STATUS_NONFINITE and is binned as 0. */
int hacc_bin(const hacc_mesh *mesh, const float *x, const float *y, const float *z,
             const float *dx, const float *dy, const float *dz, const float *m,
             const hacc_binned *out, void *ws, size_t ws_bytes, uint32_t *status, void *stream);

/* Same as hacc_bin (absolute positions, no displacements), for callers that
 * cannot allocate device memory: a plugin
 * whose host application owns every device allocation through its own pool,
 * or code running where cudaMalloc is not allowed or would stall the device
 * (inside a captured stream, a host callback, a real-time loop).  The scratch
 * space that hacc_bin takes as `ws` is instead one fixed array that the
 * library places in device memory when it is loaded: HACC_BIN_NOALLOC_BYTES
 * (9 MiB); every device that loads the library keeps it until the process
 * exits.  A problem fits when hacc_bin_workspace_size(mesh) is at most that,
 * about 30 bytes per particle whatever the number of cells (262,144
 * particles fit, 400,000 do not); larger problems return HACC_ERR_CAPACITY
 * (use hacc_bin with a workspace).  The caller still passes the inputs and the outputs in `out`;
 * nothing is allocated or freed, by this library or any other.
 * The first call on each device looks up the array's device address, with
 * that device current; make that first call before any stream capture (a
 * first call on a stream that is being captured returns HACC_ERR_INVALID and
 * leaves the capture intact).
 * All calls share the one array: calls whose work overlaps on the GPU (on
 * different streams, or from several host threads) race and must be
 * serialised by the caller.  Each call clears the scratch it relies on, so
 * one call's leftovers never change the next call's result.
 * The paper has no counterpart: this is an interface for embedding. */
#define HACC_BIN_NOALLOC_BYTES ((size_t)9 << 20)
int hacc_bin_noalloc(const hacc_mesh *mesh, const float *x, const float *y, const float *z,
                     const float *m, const hacc_binned *out, uint32_t *status, void *stream);

/* Upper bound of the task count for split size T (host). */
int64_t hacc_task_capacity(const hacc_mesh *mesh, int32_t split_T);

/* Bytes of scratch that hacc_build_lists needs. */
size_t hacc_lists_workspace_size(const hacc_mesh *mesh);

/* Builds the per-cell neighbour-cell lists within the cutoff -- the
 * analogue of the paper's tree walk producing leaf-shared interaction lists
 * (Sec. III, walk minimisation; every particle of a cell shares the cell's
 * list, Sec. III) -- and the task list.  A cell c' (with periodic image) is
 * listed for cell c iff the two boxes can hold a pair closer than r_c:
 * sum_a max(0, |delta_a| - 1)^2 w^2 < r_c^2 (float64), delta = integer cell
 * offset; entries in ascending (dz, dy, dx).  Tasks cut each cell's sorted
 * range into chunks of at most split_T particles, cells ascending; task_order
 * lists them heaviest first (so that the persistent pair kernels do not end
 * on a long halo task), ties in cell order.  Also
 * counts the candidate pairs into *lists->n_pairs.  More tasks than task_cap
 * sets HACC_STATUS_CAPACITY (the surplus is not written). */
int hacc_build_lists(const hacc_mesh *mesh, const hacc_binned *binned, const hacc_lists *lists,
                     void *ws, size_t ws_bytes, uint32_t *status, void *stream);

/* ---- RCB fat-leaf tree: the paper's own list builder (Sec. III) ---------
 * An alternative to hacc_bin + hacc_build_lists whose leaves take the place
 * of the chaining-mesh cells; the pair calls (hacc_sr_force, the adjoint, the
 * potential, hacc_count_pairs) take its output unchanged. */
#define HACC_RCB_QBITS 21     /* quantisation: 2^21 steps per box side */
#define HACC_RCB_MAX_DEPTH 64 /* largest accepted max_depth */

typedef struct hacc_tree {
    int32_t leaf_max;    /* in: a group of more than leaf_max particles is split, >= 1 */
    int32_t max_depth;   /* in: groups at this depth become leaves whatever their size,
                            0..HACC_RCB_MAX_DEPTH (roots have depth 0) */
    int64_t leaf_cap;    /* in: capacity of the leaf and node arrays, in leaves (N suffices) */
    int32_t *n_leaves;   /* device scalar out */
    int32_t *n_nodes;    /* device scalar out: internal nodes */
    int32_t *leaf_start; /* [leaf_cap + 1] first sorted slot of each leaf, [n_leaves] = N */
    int32_t *leaf_qbox;  /* [6 leaf_cap] leaf box on the 2^21 grid of its volume: lo xyz, hi xyz */
    float *leaf_origin;  /* [4 leaf_cap] (x, y, z, 0): float32 of lo L / 2^21 (float64 product) */
    int32_t *node_qbox;  /* [6 leaf_cap] boxes of the internal nodes, same layout */
    int32_t *node_child; /* [2 leaf_cap] left, right child: node id >= 0, or -1 - leaf id */
    int32_t *root;       /* [V] root of each volume: node id, -1 - leaf id, or INT32_MIN if empty */
} hacc_tree;

/* Bytes of scratch that hacc_rcb_build needs for groups of more than leaf_max
 * particles. */
size_t hacc_rcb_build_workspace_size(const hacc_mesh *mesh, int32_t leaf_max);

/* Recursive coordinate bisection of every volume into leaves of at most
 * leaf_max particles (Sec. III: split at the centre of mass, perpendicular
 * to the longest side of the group's box, halves kept contiguous), made exact
 * in integers so the tree is reproducible bit for bit.  Per axis q =
 * floor(xw 2^21 / L), clamped to [0, 2^21), xw wrapped as in hacc_bin, the
 * product in float64; the box of a group is the min/max of its q; the split
 * axis is the longest side (lowest axis on ties), the split value the floor
 * of the mean q (equal masses: the centre of mass); a particle goes left iff
 * q <= split, the partition is stable; a group whose box is a point is
 * halved by position (cnt/2 left).  Leaves are numbered depth first, left
 * first (= by first slot).  Writes every array of `tree`, and of `out`:
 * perm, sorted4 with o = fl32(xw - origin) (float64 difference), cell_of and
 * mass_varies if not NULL; `out->cell_start` and `out->cell_origin` are not touched (point
 * them at tree->leaf_start and tree->leaf_origin for the pair calls).
 * Level-synchronous on the GPU: it SYNCHRONISES `stream` once per tree level
 * to read the number of groups left, so it cannot be captured in a CUDA
 * graph.  More leaves or nodes than leaf_cap sets HACC_STATUS_CAPACITY; a
 * non-finite coordinate sets HACC_STATUS_NONFINITE and is taken as 0. */
int hacc_rcb_build(const hacc_mesh *mesh, const float *x, const float *y, const float *z, const float *m,
                   const hacc_tree *tree, const hacc_binned *out, void *ws, size_t ws_bytes, uint32_t *status,
                   void *stream);

/* Bytes of scratch that hacc_rcb_lists needs. */
size_t hacc_rcb_lists_workspace_size(const hacc_mesh *mesh, int64_t leaf_cap, int64_t task_cap);

/* Leaf-shared interaction lists by a walk of the tree (Sec. III, walk
 * minimisation), and the tasks.  Leaf j with periodic image s is listed for
 * leaf i iff the two leaf boxes, each widened by one grid step L / 2^21 on
 * every side ([(lo - 1) L / 2^21, (hi + 2) L / 2^21], float64), come closer
 * than the volume's rcut (sum of squared gaps < rcut^2, float64); entries in
 * ascending image code (sz+1)*9 + (sy+1)*3 + (sx+1), then ascending j.  An
 * internal node is skipped when its widened box fails the same test, which
 * never drops a leaf that passes.  Writes lists->nbr_off [leaf_cap + 1] and
 * the entry count into the device int64 *n_entries; if lists->nbr_cell is
 * NULL nothing else is done (a sizing pass).  Otherwise, when the count fits
 * entry_cap, the entries, and then the tasks (each leaf cut into chunks of at
 * most split_T particles), task_order (heaviest first, as hacc_build_lists)
 * and *n_pairs; a count above entry_cap, or more tasks than task_cap, sets
 * HACC_STATUS_CAPACITY.  Requires a tree built by hacc_rcb_build on the same
 * mesh. */
int hacc_rcb_lists(const hacc_mesh *mesh, const hacc_tree *tree, const hacc_lists *lists, int64_t entry_cap,
                   int64_t *n_entries, void *ws, size_t ws_bytes, uint32_t *status, void *stream);

/* Bytes of scratch that hacc_sr_force / hacc_sr_force_adjoint need. */
size_t hacc_force_workspace_size(const hacc_mesh *mesh);

/* Short-range force (Eq. 7) on every particle, written to ax, ay, az [N] in
 * input order (overwritten).  float32 arithmetic with the cutoff applied as a
 * select inside the pair loop (the paper's fsel discussion, Sec. III),
 * rsqrt from the hardware unit, per-particle compensated accumulation.
 * Requires eps > 0 (the softening keeps the self and coincident pairs
 * finite) and p->rcut equal to the rcut the mesh was planned with. */
int hacc_sr_force(const hacc_mesh *mesh, const hacc_binned *binned, const hacc_lists *lists,
                  const hacc_sr_params *p, float *ax, float *ay, float *az,
                  const hacc_launch *launch, void *ws, size_t ws_bytes, uint32_t *status,
                  void *stream);

/* Same forces as hacc_sr_force from half the pair evaluations: each pair
 * inside the cutoff is evaluated once and applied to both particles
 * (Newton's third law; the paper's kernel instead evaluates every particle's
 * own list, Sec. III).  Each task walks its cell itself and the entries after
 * the cell in its list (lists are symmetric: a chaining-mesh cell's own
 * entry sits in the middle of its list, a tree leaf's is found by bisection
 * of its (image, leaf) order); a warp holds 32 j records
 * one per lane and rotates them, with their force partial sums, through the
 * lanes by shuffles; the partial sums are added to float64 per-particle
 * totals with atomics, converted to float32 at the end.  Chaining-mesh and
 * tree lists alike.  Results agree with hacc_sr_force
 * to float32 rounding but are not bitwise reproducible (the float64 sums
 * are formed in a run-dependent order).  Workspace: hacc_force_workspace_size. */
int hacc_sr_force_symmetric(const hacc_mesh *mesh, const hacc_binned *binned, const hacc_lists *lists,
                            const hacc_sr_params *p, float *ax, float *ay, float *az,
                            const hacc_launch *launch, void *ws, size_t ws_bytes, uint32_t *status,
                            void *stream);

/* hacc_sr_force_adjoint with each pair evaluated once: the pair's terms of
 * dL/dx are antisymmetric (J(d) is even in d), so the j side receives minus
 * the i side's: one vector sum W per particle when gm is NULL, the factored
 * sums U, V, X, G of the gather adjoint otherwise (float64 totals by atomics,
 * as hacc_sr_force_symmetric).
 * Same arguments and outputs as hacc_sr_force_adjoint; chaining-mesh or
 * tree lists; not bitwise reproducible.  Not in the paper. */
int hacc_sr_force_adjoint_symmetric(const hacc_mesh *mesh, const hacc_binned *binned,
                                    const hacc_lists *lists, const hacc_sr_params *p, const float *gax,
                                    const float *gay, const float *gaz, float *gx, float *gy, float *gz,
                                    float *gm, const hacc_launch *launch, void *ws, size_t ws_bytes,
                                    uint32_t *status, void *stream);

/* Vector-Jacobian product of hacc_sr_force (not in the paper).  Given
 * lam = dL/da (gax, gay, gaz, [N] input order) returns, in input order,
 *   gx_i = dL/dx_i = sum_j [m_i J(d_ij) lam_j - m_j J(d_ij) lam_i],
 *   J(d) = f_SR(s) I + 2 f_SR'(s) d d^T,
 *   gm_i = dL/dm_i = -sum_j f_SR(s_ij) d_ij . lam_j        (gm may be NULL),
 * recomputing every pair term (nothing is stored by the forward call).  With
 * gm NULL each pair adds J(d_ij) mu_ij, mu_ij = m_i lam_j - m_j lam_i, to one
 * vector sum; with gm the kernel keeps the sums U = sum f lam_j, V = sum m_j f,
 * X = sum 2 f' (m_i d.lam_j - m_j d.lam_i) d and G (gx = m_i U - lam_i V + X). */
int hacc_sr_force_adjoint(const hacc_mesh *mesh, const hacc_binned *binned,
                          const hacc_lists *lists, const hacc_sr_params *p, const float *gax,
                          const float *gay, const float *gaz, float *gx, float *gy, float *gz,
                          float *gm, const hacc_launch *launch, void *ws, size_t ws_bytes,
                          uint32_t *status, void *stream);

/* Short-range potential of every particle, phi [N] in input order:
 *   phi_i = sum_{j != i, s_ij < r_c^2} m_j V(s_ij),
 *   V(s) = (r_c^2 + eps)^(-1/2) - (s + eps)^(-1/2) + [P(r_c^2) - P(s)] / 2,
 *   P(s) = sum_k c_k s^(k+1) / (k+1),
 * the integral of the force law of Eq. 7 (F = -grad V) that vanishes at the
 * cutoff; the energy of the short-range sub-cycles of Eq. 6 is then
 * sum m v^2/2 + sum m phi / 2 (hacc_moments).  Same arithmetic, staging and
 * arguments as hacc_sr_force. */
int hacc_sr_potential(const hacc_mesh *mesh, const hacc_binned *binned, const hacc_lists *lists,
                      const hacc_sr_params *p, float *phi, const hacc_launch *launch, void *ws,
                      size_t ws_bytes, uint32_t *status, void *stream);

/* Counts, into the device int64 *out, the ordered pairs (j != i) that the
 * pair kernels find inside the cutoff: s + eps < r_c^2 + eps evaluated in
 * float32 on the cell-relative offsets exactly as hacc_sr_force evaluates it
 * (the paper's "short-range condition", Sec. III).  With the candidate count
 * of hacc_build_lists it gives the lists' efficiency.  A reporting tool, not
 * a hot path (one i per lane, j straight from global memory). */
int hacc_count_pairs(const hacc_mesh *mesh, const hacc_binned *binned, const hacc_lists *lists,
                     const hacc_sr_params *p, int64_t *out, void *stream);

/* Kick and optional drift of the split-operator step (Eq. 6):
 *   v <- v + dt_kick a;  then, if x != NULL, x <- x + dt_drift v (new v),
 * the drift computed in float64 and rounded once to float32.  If `mesh` is
 * non-NULL the drifted positions are wrapped into [0, L) of their volume.
 * Arrays [N] in input order; x, y, z may be NULL (kick only); ax, ay, az may
 * be NULL (the stream map alone: v is read, never written); not both. */
int hacc_kick(const hacc_mesh *mesh, int64_t N, float *vx, float *vy, float *vz, const float *ax,
              const float *ay, const float *az, float dt_kick, float *x, float *y, float *z,
              float dt_drift, void *stream);

/* Stream map on the binned particles, for re-binning amortisation over
 * short-range sub-cycles (Eq. 6): every sorted record's cell-relative offset
 * moves by dt v of its particle (o <- fma(dt, v, o) in float32; v [N] in input
 * order, looked up through perm), so the pair calls can run again without
 * re-binning.  The lists stay complete while every particle stays within
 * skin/2 of its cell box, i.e. if they were built for r_c + skin (plan the
 * mesh with rcut = r_c + skin and cell_min >= r_c + skin): an offset outside
 * [-(w + skin)/2, (w + skin)/2) (offsets are taken from the cell centre) on
 * any axis sets HACC_STATUS_SKIN, after which the
 * caller must re-bin.  The input-order positions are not touched (drift them
 * with hacc_kick and no accelerations).  Not in the paper, whose sub-cycles
 * rebuild the tree walk each time. */
int hacc_drift_offsets(const hacc_mesh *mesh, const hacc_binned *binned, const float *vx, const float *vy,
                       const float *vz, float dt, float skin, uint32_t *status, void *stream);

/* Bytes of scratch that hacc_moments needs. */
size_t hacc_moments_workspace_size(int64_t N);

/* Global reductions, in a fixed order (deterministic):
 *   out[0..2] = sum m v,  out[3..5] = sum m a  (zero by Newton's third law),
 *   out[6] = sum m |v|^2 / 2,  out[7] = sum m |a|,
 *   out[8] = sum m phi / 2 (the short-range potential energy; each pair once).
 * Each particle's terms and each thread's partial sums (groups of four
 * consecutive particles at a fixed stride) are formed in double-float
 * arithmetic on the float32 pipe
 * (exact products by fma, TwoSum accumulation, about 48 significant bits;
 * |a| by a float32 root plus one Newton correction), and the per-thread sums
 * are reduced in float64.  v (vx, vy, vz), a (ax, ay, az) and phi may each be
 * NULL (their sums are then 0); v and a are all three components or none.
 * out: device double[9]. */
int hacc_moments(int64_t N, const float *m, const float *vx, const float *vy, const float *vz,
                 const float *ax, const float *ay, const float *az, const float *phi, double *out,
                 void *ws, size_t ws_bytes, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* HACC_SR_H */

/*
 * meshloop -- C ABI of the GB300 (sm_103a) library for locality-optimised
 * indirect-increment mesh loops, after Sulyok, Balogh, Reguly and Mudalige,
 * "Locality Optimized Unstructured Mesh Algorithms on GPUs" (2018).
 *
 * Model (Sec. 1.1.1): a mesh is a collection of sets; a map gives, for every
 * element of a from-set, a fixed number (the arity) of indices into a to-set;
 * data live on sets.  A loop runs over a from-set, reads data directly on it
 * or through one level of maps, and may INCREMENT data through a map.  The
 * result must not depend on iteration order, up to rounding.
 *
 * Execution (Sec. 2.2, Algorithm 1): iterations are grouped into blocks of at
 * most S (one CUDA thread block each).  Each block stages the to-set data it
 * touches (its "footprint") in shared memory, computes every iteration from
 * shared memory, applies its increments to shared memory one thread colour at
 * a time, and writes each footprint point back to global memory once.
 * Blocks of one block colour never share a written point, so a launch per
 * block colour needs no atomics (two-layer or hierarchical colouring).
 * Baselines from Sec. 2.1: global colouring (one launch per iteration
 * colour, direct global read-modify-write) and atomics.
 *
 * Planning (Sec. 2.3): optional reverse Cuthill-McKee reordering (a
 * bandwidth-reducing BFS ordering in the spirit of GPS), partitioning of the
 * iterations into compact blocks of at most S' = floor(S / l) (Eq. 1),
 * data-point reordering by the set of accessing blocks, first-fit block and
 * thread colouring.
 *
 * Conventions used by every call below:
 *  - Return value: MP_OK (0) or a negative MP_E* code; mp_error_string()
 *    names it.  A failing call leaves its outputs unspecified but frees
 *    whatever it allocated.
 *  - Host pointers are read during the call only; the caller keeps them.
 *  - Data pointers passed to loop_* calls are DEVICE pointers of the
 *    current CUDA device, owned by the caller, 16-byte aligned, in PLAN
 *    numbering (mesh_plan_perm gives the permutations).  Data are stored
 *    either array-of-structures (x[node][2]) or structure-of-arrays
 *    (x[2][node]) as chosen by mp_plan_opts.layout; dtype selects double or
 *    float storage and arithmetic.
 *  - Increments are "+=": the caller zeroes an increment target first.
 *  - Loop calls are asynchronous on the given stream (0 = legacy default)
 *    and never synchronise the device.  The first loop call on a plan
 *    uploads its tables (cudaMalloc + cudaMemcpy, synchronous); call
 *    mesh_plan_upload() first when the loop will be captured in a graph.
 */
#ifndef MESHLOOP_H
#define MESHLOOP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status codes */
#define MP_OK 0
#define MP_EINVAL (-1)     /* null or misaligned pointer, bad arity/size/option        */
#define MP_EMAPRANGE (-2)  /* a map index is outside [0, to_size)                      */
#define MP_ECOLORS (-3)    /* more than MP_MAX_BLOCK_COLORS block colours (Sec. 3.1.5)  */
#define MP_ESMEM (-4)      /* a block footprint exceeds shared memory (Sec. 3.1.5)      */
#define MP_ECUDA (-5)      /* a CUDA runtime call failed                               */
#define MP_ETIMEOUT (-6)   /* a bounded device-side wait gave up                       */
#define MP_ENOMEM (-7)     /* host allocation failed                                   */
#define MP_EPLAN (-8)      /* plan does not fit the loop (maps, colouring, layout)     */
#define MP_EIO (-9)        /* plan file could not be read or written                   */
#define MP_ETOOBIG (-10)   /* size exceeds the fixed static scratch of an allocation-free
                              entry point                                                */

#define MP_MAX_BLOCK_COLORS 256  /* limit of the paper's library, Sec. 3.1.5        */
#define MP_MAX_THREAD_COLORS 64
#define MP_MAX_MAPS 4
#define MP_MAX_TOSETS 2

/* ------------------------------------------------------------- options */
enum { MP_REORDER_NONE = 0, MP_REORDER_RCM = 1, MP_REORDER_PARTITION = 2 };
enum { MP_COLOR_HIER = 0, MP_COLOR_GLOBAL = 1, MP_COLOR_ATOMIC = 2, MP_COLOR_TWOSTEP = 3 };
/* MP_COLOR_TWOSTEP (Sec. 2.1, the temporary-array method): a first kernel
 * writes every iteration's increments to a scratch array of from_size x
 * arity x dim values; a second kernel gathers them per point of the written
 * to-set through the inverse map (fixed order, deterministic).  Plans with
 * exactly one written map; the library allocates the scratch on the first
 * loop call and frees it with the plan.                                  */
enum { MP_LAYOUT_AOS = 0, MP_LAYOUT_SOA = 1 };
enum { MP_F64 = 0, MP_F32 = 1, MP_F64_DW = 2 };
/* MP_F64_DW: FP64 data, arithmetic in double-word (pairs of FP32, ~48-bit
 * significand, FP32's exponent range) on the FP32 pipes; results agree with
 * FP64 to ~1e-13 relative while the values the loop forms (inputs, their
 * products and the fluxes) stay within about 1e-30..1e38 in magnitude:
 * zeros are exact, smaller values lose relative precision gradually
 * (subnormal FP32 low parts), larger ones overflow.  Offered by
 * loop_res_calc, loop_adjoint, loop_elem_assemble and loop_face_flux with
 * HIER plans (res_calc and hex assembly: gather increments by default,
 * MP_STAGED_SIMPLE for thread colours; hex: blocks of at most 256 threads;
 * face flux: at most 128), and by loop_res_calc, loop_adjoint and
 * loop_elem_assemble with GLOBAL and ATOMIC plans (the Sec. 2.1 baselines
 * in the same arithmetic: FP64 read-add-write of the incremented data per
 * colour, or FP64 atomicAdd).                                            */

/* One map of the loop: from the loop's iteration set (set id 0) to the
 * caller's set `to_set` (ids >= 1; maps with the same id share a to-set).
 * idx is host memory, from_size x arity, row-major, int32.               */
typedef struct {
    int32_t to_set;
    int32_t arity;     /* 1..8                                            */
    int64_t to_size;   /* number of points in the to-set                  */
    const int32_t *idx;
    int32_t written;   /* 1: the loop increments data through this map   */
    int32_t pad_;
} mp_map;

/* Planner options (Sec. 2.3 tuning parameters). */
typedef struct {
    int32_t block_size;  /* S: launched threads per block, 32..1024, multiple of 32  */
    int32_t reorder;     /* MP_REORDER_*                                             */
    int32_t coloring;    /* MP_COLOR_*                                               */
    int32_t layout;      /* MP_LAYOUT_*                                              */
    double imbalance;    /* l of Eq. 1 (default 1.001); S' = floor(S / l)            */
    double eps;          /* epsilon of Eq. 2 (default 0), reported through l'        */
    int32_t primary_map; /* map whose to-set is RCM-ordered; -1 = first written map  */
    int32_t data_reorder;/* 1: reorder to-set points by accessing blocks (Sec. 2.3.2);
                            -1: default (on with MP_REORDER_PARTITION)              */
    int32_t staged;      /* MP_STAGED_* implementation of HIER loops; -1: the loop's
                            default (hex assembly, whose 3D blocks need ~10 thread
                            colours: MP_STAGED_SMEM_ATOMIC in FP32 and FP64;
                            MP_STAGED_GATHER for res_calc in every
                            arithmetic, the double-word hex assembly and adjoint,
                            and the increment-only loops; MP_STAGED_SIMPLE
                            otherwise)                                               */
    int32_t recolor;     /* HIER: after the first-fit block colouring, empty the last
                            colours when they hold few blocks (at most 1/32 of them)
                            by moving each of their blocks to an earlier colour
                            whose conflicting blocks (at most two) can themselves
                            move to a third colour, by a two-colour interchange,
                            or split into pieces that fit earlier colours: fewer,
                            fuller launches.  Plans with more than 64 block
                            colours keep first fit.
                            0: off (the first-fit colouring alone), 1: on,
                            -1: default (on)                                         */
    const int32_t *block_of; /* optional, host, from_size entries: caller-defined
                            blocks (e.g. handcrafted shapes on a structured mesh,
                            Sec. 3.1.6).  Iterations with equal values form one block
                            (ascending value order, iterations ascending inside); no
                            reordering or partitioning is applied; each block must
                            hold at most block_size iterations (else MP_EINVAL).     */
} mp_plan_opts;

/* Fill opts with defaults: S = 512, PARTITION, HIER, AOS, l = 1.001,
 * staged = -1 (the loop's default). */
void mp_plan_opts_default(mp_plan_opts *opts);

typedef struct mp_plan mp_plan;

/* Plan statistics (Sec. 3.1's counters). reuse[t] = accesses to to-set t
 * through staged maps / staged footprint points, summed over blocks (the
 * paper's data reuse factor, Sec. 3.1).                                  */
typedef struct {
    int64_t from_size;
    int32_t nblocks;
    int32_t nblock_colors;     /* block colours (HIER) or iteration colours (GLOBAL)  */
    int32_t max_thread_colors;
    int32_t block_size;        /* S                                                  */
    int32_t sprime;            /* S' of Eq. 1                                         */
    int32_t ntosets;
    double lprime;             /* l' of Eq. 2                                         */
    double mean_thread_colors;
    double reuse[MP_MAX_TOSETS];
    double reuse_all;          /* over all staged maps                               */
    int64_t footprint_total[MP_MAX_TOSETS];
    int32_t footprint_max[MP_MAX_TOSETS];
    int32_t to_set_id[MP_MAX_TOSETS];
    int64_t to_set_size[MP_MAX_TOSETS];
    int64_t plan_bytes;        /* device bytes of the plan tables                     */
    double seconds_total, seconds_reorder, seconds_partition, seconds_color;
} mp_plan_stats;

/* Build a plan for a loop over a from-set of from_size iterations with the
 * given maps (Sec. 2.3; reordering, partitioning, colouring).  Host only;
 * touches no GPU.  *out is owned by the caller: mesh_plan_destroy().
 * Errors: MP_EINVAL, MP_EMAPRANGE, MP_ECOLORS, MP_ENOMEM.                */
int mesh_plan_build(const mp_map *maps, int32_t nmaps, int64_t from_size, const mp_plan_opts *opts,
                    mp_plan **out);
/* Free a plan and its device tables (NULL is a no-op).  The plan is the
 * reusable product of the one-off reordering and colouring (Sec. 2.3.2);
 * it must not be in use by a loop call still queued on a stream.        */
void mesh_plan_destroy(mp_plan *plan);
/* Plan statistics (Sec. 3.1's block counts, colour counts and data reuse).
 * Errors: MP_EINVAL (null argument).                                    */
int mesh_plan_query(const mp_plan *plan, mp_plan_stats *stats);

/* new_to_old permutation of set `set_id` (0 = the from-set, else a to-set
 * id of the maps): new_to_old[new] = old, length = the set's size.  The
 * renumbering of Sec. 2.3.1 (reordering of the primary to-set and the
 * iterations) and Sec. 2.3.2 (data points by accessing blocks): callers
 * move their data into plan numbering with it.  new_to_old is host memory
 * of the set's size, owned by the caller.  Errors: MP_EINVAL (null
 * argument or unknown set id).                                           */
int mesh_plan_perm(const mp_plan *plan, int32_t set_id, int32_t *new_to_old);

/* Copy one host plan table into out (capacity `cap` elements of the
 * table's type; *count receives the length).  Tables:
 *   MP_TAB_BLOCK_OFFSETS  int32[nblocks+1]  iteration range of each block
 *   MP_TAB_COLOR_OFFSETS  int32[ncolors+1]  block (HIER) or iteration (GLOBAL)
 *                                           range of each colour
 *   MP_TAB_BLOCK_COLOR    int32[nblocks]
 *   MP_TAB_THREAD_COLOR   int32[from_size]  thread colour of each iteration
 *   MP_TAB_MAP            int32[from_size*arity] map `arg` in plan numbering
 *   MP_TAB_FOOTPRINT      int32[...]  HIER: all blocks' footprint lists (plan
 *                                     numbering), to-set slot 0 first
 *   MP_TAB_FP_START       int32[nblocks*MP_MAX_TOSETS] HIER: offset of each
 *                                     block's list per slot in MP_TAB_FOOTPRINT
 *   MP_TAB_FP_COUNT       int32[nblocks*MP_MAX_TOSETS] HIER: list lengths
 *   MP_TAB_LOCAL_MAP      int32[from_size*stride] HIER: block-local index of
 *                                     every map slot (maps in order, padded
 *                                     to stride = 4, 8 or 16 entries)
 *   MP_TAB_GATHER         int32[len(MP_TAB_FOOTPRINT) * W] HIER: per
 *                                     footprint point a row of W (4, 8 or 16;
 *                                     count 0 when some point of a block has
 *                                     more than 16 increments) entries: block-
 *                                     local iteration * 16 + map slot of each
 *                                     increment of the point, ascending, then
 *                                     -1 padding
 *   MP_TAB_INV_OFFSETS    int32[to_size+1] TWOSTEP: range of each point of
 *                                     the written to-set in MP_TAB_INV_INDEX
 *   MP_TAB_INV_INDEX      int32[from_size*arity] TWOSTEP: item*arity + slot
 * Iterations are in plan numbering.                                       */
enum { MP_TAB_BLOCK_OFFSETS = 0, MP_TAB_COLOR_OFFSETS = 1, MP_TAB_BLOCK_COLOR = 2,
       MP_TAB_THREAD_COLOR = 3, MP_TAB_MAP = 4, MP_TAB_FOOTPRINT = 5, MP_TAB_FP_START = 6,
       MP_TAB_FP_COUNT = 7, MP_TAB_LOCAL_MAP = 8, MP_TAB_INV_OFFSETS = 9, MP_TAB_INV_INDEX = 10,
       MP_TAB_GATHER = 11 };
int mesh_plan_table(const mp_plan *plan, int32_t table, int32_t arg, int32_t *out, int64_t cap,
                    int64_t *count);

/* Renumber a map given new_to_old permutations of its from-set and to-set
 * (either may be NULL for identity) and sort nothing else:
 *   out[i][k] = old_to_new_to[idx[from_perm[i]][k]].                     */
int mesh_map_renumber(const int32_t *idx, int64_t from_size, int32_t arity, const int32_t *from_perm,
                      const int32_t *to_perm, int64_t to_size, int32_t *out);

/* Fuse the HIER plans of n meshes of one loop (same maps, AoS layout) into
 * one plan over their disjoint union, for batched execution: the data of
 * mesh k follow those of meshes 0..k-1 in every set (concatenated arrays,
 * each mesh in its own plan numbering).  The fused block-descriptor table
 * groups every mesh's blocks by colour, so a loop call on the fused plan
 * runs the whole batch with one launch per colour phase.  Meshes keep their
 * own block size, reordering and colouring; launches use the largest block
 * size.  mesh_plan_perm on the fused plan returns the concatenated
 * permutations (offset by the mesh's base).  The inputs are not retained.
 * Errors: MP_EINVAL (a plan is not HIER/AoS or the maps differ), MP_ENOMEM.*/
int mesh_batch_build(const mp_plan *const *plans, int32_t n, mp_plan **out);

/* Copy the plan's tables to the current device (synchronous).  Idempotent.*/
int mesh_plan_upload(mp_plan *plan);

/* Select the staged implementation (MP_STAGED_*, or -1 for each loop's
 * default) of an existing HIER plan: the tables do not depend on it.  Not
 * while a loop call on the plan is being issued from another thread.
 * Errors: MP_EINVAL (null plan or value out of range).                    */
int mesh_plan_set_staged(mp_plan *plan, int32_t staged);

/* Serialise / restore a plan (reordering is a reusable one-off, Sec. 2.3.2).*/
int mesh_plan_save(const mp_plan *plan, const char *path);
int mesh_plan_load(const char *path, mp_plan **out);

/* --------------------------------------------------------------- loops */
/* Airfoil-style flux loop res_calc (Sec. 3.1.1): over interior edges,
 * reading x (2 per node) on 2 nodes and q (4), adt (1) on 2 cells, and
 * incrementing res (4 per cell) on the 2 cells: res[c1] += f, res[c2] -= f
 * with the central flux plus scalar dissipation
 *   f = (F(q1).n + F(q2).n)/2 + eps (adt1 + adt2)/2 (q1 - q2),
 *   n = (y_a - y_b, x_b - x_a), F.n the 2D Euler normal flux, gamma = gam.
 * The plan must have maps {edge->node (arity 2), edge->cell (arity 2,
 * written)} in this order; edge->node may be marked written (the adjoint's
 * plan, so that forward and adjoint share one numbering).  The colouring of the plan selects the variant:
 * HIER (staged two-layer, the product), GLOBAL or ATOMIC.  dtype MP_F64,
 * MP_F32, or MP_F64_DW (HIER plans only; FP64 data, double-word arithmetic).
 * x: [nodes][2], q: [cells][4], adt: [cells], res: [cells][4] (AoS; SoA
 * transposes each).  stream is a cudaStream_t.
 * HIER plans run one launch per block colour; every launch after the first
 * is a programmatic dependent launch (it stages q, adt and x while the
 * previous colour finishes and reads res after it), unless the environment
 * variable MESHLOOP_NO_PDL is set.                                        */
int loop_res_calc(const mp_plan *plan, int32_t dtype, const void *x, const void *q, const void *adt,
                  void *res, double gam, double eps, void *stream);

/* res_calc with HOST buffers (pinned host memory for asynchronous copies;
 * pageable memory works but the copies then block the calling thread).
 * Arguments and layout as loop_res_calc, all four arrays in host memory.
 * Enqueues on `stream`, after the work already on it: the copy of x, q,
 * adt and res into library-owned device buffers (chunks over four internal
 * copy streams), the loop, and the copy of res back into the caller's array
 * (chunks over two internal streams), joined back into `stream`.  The result is
 * in `res` once `stream` has completed; the host arrays must not be
 * modified before then.  Two device buffer slots (4 arrays each, owned by
 * the plan, freed with it) alternate between calls, so consecutive calls
 * issued on two different streams overlap one call's copies with the
 * other's loop.  Not in the paper: the end-to-end entry point of an
 * application whose data live on the host.  Errors as loop_res_calc, plus
 * MP_ECUDA for allocation, stream or copy failures.                       */
int loop_res_calc_host(const mp_plan *plan, int32_t dtype, const void *x, const void *q, const void *adt,
                       void *res, double gam, double eps, void *stream);

/* Implementations of the staged two-layer (HIER) loops, chosen per plan
 * with mp_plan_opts.staged:
 *  MP_STAGED_SIMPLE: Algorithm 1 as printed, one block per CTA, increments
 *    applied one thread colour at a time (res prefetched at staging, so the
 *    write-back is a store);
 *  MP_STAGED_PIPELINED: res_calc FP64/FP32 only: persistent CTAs walk
 *    several blocks of a colour, and asynchronous copies (cp.async) stage
 *    block k+1's footprint while block k is computed (blocks of at most 512
 *    threads whose two stages fit shared memory; otherwise SIMPLE);
 *  MP_STAGED_SMEM_ATOMIC: as SIMPLE, but increments go to shared memory with
 *    atomic adds instead of one pass per thread colour (one barrier; the
 *    order of additions, and so the rounding, is not fixed).  Not for the
 *    double-word res_calc or the adjoint, which run SIMPLE instead.
 * Block colouring orders the write-back in every variant.                */
enum { MP_STAGED_SIMPLE = 1, MP_STAGED_PIPELINED = 0, MP_STAGED_SMEM_ATOMIC = 2, MP_STAGED_GATHER = 3,
       MP_STAGED_INC_ONLY = 4, MP_STAGED_INC_ONLY_GATHER = 5, MP_STAGED_WARP_AGG = 6,
       MP_STAGED_PERSISTENT = 7 };
/* MP_STAGED_PERSISTENT: res_calc (native FP64 and FP32, gather increments)
 * in ONE cooperative launch per call instead of one launch per block
 * colour: a grid of resident CTAs walks the block-descriptor table colour
 * by colour (each CTA takes the colour's next block from a counter), and
 * the CTAs meet at a grid-wide barrier between colours.  The barrier's wait is bounded (1
 * s): if it runs out the CTAs return, the result is invalid and
 * mp_check_device_status reports MP_ETIMEOUT; nothing hangs.  The barrier
 * and block counters belong to the plan: calls on one plan must not
 * overlap.  On a
 * fused batch plan (mesh_batch_build) this runs every mesh of the batch in
 * one launch.  Other dtypes run MP_STAGED_GATHER.                        */
/* MP_STAGED_WARP_AGG: warp-aggregated increments: lanes of a warp that
 * increment the same point combine their values with a segmented shuffle
 * tree (match.any groups) and one lane adds the sum with a shared-memory
 * atomic; one barrier, order across warps not fixed.  res_calc (native
 * FP64 and FP32) and hex assembly.                                        */
/* MP_STAGED_INC_ONLY(_GATHER): shared memory caches only the increments (and
 * the current values they add to); the loop reads its indirect inputs
 * through L1/L2 instead of staging them (Sec. 3.1.5: for loops whose
 * per-point inputs exceed shared memory).  Thread-coloured or gather
 * increments.  loop_face_flux.                                            */
/* MP_STAGED_GATHER: no thread colours: each thread stores its iteration's
 * increments in shared memory, one barrier, then every footprint point sums
 * the increments of its iterations in the block (block-local inverse map,
 * fixed order: deterministic) and writes back once.  res_calc (native and
 * double-word; native FP32 blocks of more than 256 edges, a multiple of
 * 64, run two edges per thread), hex assembly and the adjoint (double-
 * word), the increment-only loops and the face flux.                      */

/* Far-field boundary flux bres_calc over boundary edges: with
 * q_b = (q_c + qinf)/2,  res[c] += F(q_b).n + eps adt_c (q_c - qinf).
 * Plan maps {bedge->node (2, read), bedge->cell (1, written)}; colouring
 * GLOBAL or ATOMIC or HIER.  qinf: 4 host doubles.                       */
int loop_bres_calc(const mp_plan *plan, int32_t dtype, const void *x, const void *q, const void *adt,
                   void *res, const double *qinf, double gam, double eps, void *stream);

/* adt_calc over cells (read-only indirection through cell->node[4], corners
 * counter-clockwise): adt = sum over the 4 sides of
 *   (|u dy - v dx| + c sqrt(dx^2 + dy^2)) / cfl,  c = sqrt(gam p / rho).
 * Plan maps {cell->node (4, read)}; any colouring (none is needed).       */
int loop_adt_calc(const mp_plan *plan, int32_t dtype, const void *x, const void *q, void *adt,
                  double gam, double cfl, void *stream);

/* save_soln + update, direct loops over ncell cells in the given layout:
 *   loop_save_soln: qold = q
 *   loop_update:    d = res/adt (in FP64), q = qold - d, res = 0,
 *                   *rms_dev (a device double) += sum of d^2 in FP64.
 * The sum is deterministic (fixed-order two-pass reduction in plan-free
 * scratch owned by the library; calls on one device must not overlap).  */
int loop_save_soln(int64_t ncell, int32_t dtype, int32_t layout, const void *q, void *qold,
                   void *stream);
int loop_update(int64_t ncell, int32_t dtype, int32_t layout, const void *qold, void *q, void *res,
                const void *adt, double *rms_dev, void *stream);

/* Allocation-free variant of loop_update (the paper has no counterpart).
 * Same arguments as loop_update, and the same q and res bit for bit; the
 * residual sum is deterministic from run to run, but its partial sums are
 * grouped differently from loop_update's (one per CTA of 2048 cells), so
 * it may differ from loop_update's in the last bits.  Its scratch (one FP64
 * partial sum per CTA) is a fixed static device array of
 * MP_NOALLOC_MAX_PARTIALS doubles inside the library instead of memory
 * obtained from cudaMalloc, so the call never allocates or frees device
 * memory.  It is meant for callers that cannot allocate: host
 * applications that reserve all device memory up front in their own pool,
 * or that forbid device allocation (and the implicit device synchronisation
 * cudaMalloc may cause) once they are running.
 * Limits and behaviour:
 *  - ncell may be at most MP_NOALLOC_MAX_CELLS (2048 cells per partial);
 *    larger sizes return MP_ETOOBIG before anything is launched.
 *  - The first call on each device looks up the device address of the
 *    static array (cudaGetSymbolAddress) with that device current; make that
 *    first call before any stream capture.  The address is kept for the
 *    life of the process: do not reset the device's primary context
 *    (cudaDeviceReset) after that first call.
 *  - Every device that loads the library holds the array until exit.  All
 *    calls share it and it keeps the last call's partial sums; each call
 *    overwrites every entry it reads, so nothing needs clearing, but calls
 *    whose executions overlap on the GPU (other streams, other threads) race
 *    on it: serialise them.                                                 */
#define MP_NOALLOC_MAX_PARTIALS 4096
#define MP_NOALLOC_CELLS_PER_PARTIAL 2048
#define MP_NOALLOC_MAX_CELLS ((int64_t)MP_NOALLOC_MAX_PARTIALS * MP_NOALLOC_CELLS_PER_PARTIAL)
int loop_update_noalloc(int64_t ncell, int32_t dtype, int32_t layout, const void *qold, void *q, void *res,
                        const void *adt, double *rms_dev, void *stream);

/* Hex assembly (Sec. 3.1.4's IntegrateStressForElems access pattern): over
 * hex8 elements read x, v (3 per node) on 8 nodes and sig (3, direct),
 * write vol (direct) and increment f (3 per node) on the 8 nodes, with the
 * one-point hex8 stress force -diag(sig) B_i and Flanagan-Belytschko
 * hourglass force (coefficient kappa).  Corner order of elem->node:
 * (-,-,-),(+,-,-),(+,+,-),(-,+,-),(-,-,+),(+,-,+),(+,+,+),(-,+,+).
 * Plan maps {elem->node (8, written)}.  x, v, f: [nodes][3];
 * sig: [elems][3]; vol: [elems].                                         */
int loop_elem_assemble(const mp_plan *plan, int32_t dtype, const void *x, const void *v,
                       const void *sig, void *f, void *vol, double kappa, void *stream);

/* Adjoint of res_calc with x, q, adt fixed (adt not differentiated):
 *   q_bar += (d res/d q)^T res_bar,  x_bar += (d res/d x)^T res_bar.
 * Both maps are written, so the plan has maps {edge->node (2, written),
 * edge->cell (2, written)}.  dtype MP_F64, MP_F32 or MP_F64_DW.  HIER
 * plans sum each cell's and node's increments through the gather rows by
 * default (a fixed order, deterministic; MP_STAGED_SIMPLE for thread
 * colours); GLOBAL and ATOMIC as loop_res_calc, in every dtype.         */
int loop_adjoint(const mp_plan *plan, int32_t dtype, const void *x, const void *q, const void *adt,
                 const void *res_bar, void *q_bar, void *x_bar, double gam, double eps,
                 void *stream);

/* Increment-only edge loop with the access pattern of Volna's
 * SpaceDiscretization (Sec. 3.1.2): per edge 7 values and 1 integer read
 * directly, per cell 1 value read and 4 incremented.  With the edge's
 * direct data d = (F0, F1, F2, P, L, nx, ny) (flux, pressure, length, unit
 * normal out of its first cell):
 *   w = L (F0, F1 + P nx, F2 + P ny, P)
 *   res[c1] -= inv_area[c1] w;  res[c2] += inv_area[c2] w  unless eflag = 1
 * (a boundary edge lists its one cell twice and has eflag 1).
 * Plan: maps {edge->cell (2, written)}; HIER (gather increments by
 * default, MP_STAGED_SIMPLE for thread colours), GLOBAL, ATOMIC or TWOSTEP
 * (owner computes: one launch over the cells, each summing its edges'
 * increments recomputed from their direct data through the plan's inverse
 * map; no temporary array, no atomics, deterministic).  dtype MP_F32
 * (the paper's precision for this loop) or MP_F64.  edata [edges][7] (SoA
 * [7][edges]), eflag int32 [edges], inv_area [cells], res [cells][4] (SoA
 * [4][cells]); all device memory in plan numbering, 16-byte aligned.
 * Errors: MP_EINVAL (dtype, null or misaligned pointer), MP_EPLAN (plan
 * shape), MP_ECUDA.                                                      */
int loop_space_disc(const mp_plan *plan, int32_t dtype, const void *edata, const int32_t *eflag,
                    const void *inv_area, void *res, void *stream);

/* Increment-only cell loop with the access pattern of BookLeaf's
 * getacc_scatter (Sec. 3.1.3): per cell 17 values read directly,
 * (rho, m[4], w[4], fx[4], fy[4]); node k of the cell (cell->node order) gets
 *   nd[n_k] += (m_k, rho w_k, fx_k, fy_k).
 * Plan: maps {cell->node (4, written)}; HIER (block size <= 512; gather
 * increments by default, MP_STAGED_SIMPLE for thread colours), GLOBAL,
 * ATOMIC or TWOSTEP (owner computes, as loop_space_disc).  dtype MP_F64 (the paper's precision) or MP_F32.  cdata
 * [cells][17] (SoA [17][cells]), nd [nodes][4] (SoA [4][nodes]); device
 * memory in plan numbering, 16-byte aligned.  Errors as loop_space_disc. */
int loop_getacc(const mp_plan *plan, int32_t dtype, const void *cdata, void *nd, void *stream);

/* Face flux with the access pattern of miniAero's compute_face_flux
 * (Sec. 3.1.5): over interior faces of a hex mesh, 12 values read
 * directly per face, 28 read and 5 incremented on each of the 2 cells.
 * Face data (A[3] area normal from c1 into c2, xf[3] face centre, nhat[3] =
 * A/|A|, dx[3] = xc2 - xc1); cell data (Q[5] = (rho, rho u, rho v, rho w,
 * E), gradients of the primitives (rho, u, v, w, p) at 5 + 3 v + d, limiters
 * at 20 + v, centroid at 25).  Per face:
 *   V_face = V_cell + phi G (xf - xc) on each side; Rusanov flux
 *   F_inv = |A| ((F(V_1) + F(V_2))/2 - lambda (Q_2 - Q_1)/2);
 *   Newtonian viscous and heat flux F_v = (0, tau A, u_f.tau A + k grad T.A)
 *   from the cell gradients corrected along dx (T = p/rho,
 *   k = mu gam / ((gam - 1) pr));  res[c1] += F_inv - F_v, res[c2] -= it.
 * Plan: maps {face->cell (2, written)}; HIER (block size <= 256; default
 * MP_STAGED_SIMPLE: the 28 cell values staged and prepared once per cell,
 * thread-coloured increments; MP_STAGED_GATHER likewise with gather
 * increments; MP_STAGED_INC_ONLY[_GATHER] stage the increments only),
 * GLOBAL, ATOMIC or TWOSTEP (the original code's temporary array).  dtype MP_F64, MP_F32 or MP_F64_DW (HIER
 * plans, block size <= 128: FP64 data, double-word arithmetic, full staging
 * and thread-coloured increments).  fdata [faces][12], cdata
 * [cells][28], res [cells][5] (SoA: transposed); device memory in plan
 * numbering, 16-byte aligned.  Errors: MP_EINVAL (dtype, constants, null or
 * misaligned pointer, block size), MP_EPLAN (plan shape), MP_ECUDA.       */
int loop_face_flux(const mp_plan *plan, int32_t dtype, const void *fdata, const void *cdata, void *res,
                   double gam, double mu, double pr, void *stream);

/* --------------------------------------------------------------- status */
/* Name and meaning of an MP_* code (a static string; unknown codes give
 * "unknown error").  The codes include the failure modes of Sec. 3.1.5:
 * MP_ECOLORS (the 256-colour limit) and MP_ESMEM (a block footprint that
 * does not fit shared memory).                                          */
const char *mp_error_string(int code);
/* Reads (and clears) the library's device error word, where kernels record
 * what they detect while running: MP_OK, MP_ESMEM (a staged kernel found
 * its shared-memory carve-up or its block's footprint larger than the
 * launch provides, and returned without touching memory) or MP_ETIMEOUT (a
 * bounded device-side wait gave up).  Synchronises the stream.          */
int mp_check_device_status(void *stream);
/* Diagnostic of the bounded grid-wide wait that the persistent launches
 * (MP_STAGED_PERSISTENT) use between block colours; not in the paper.
 * Launches nctas resident CTAs (1 <= nctas <= the SM count, cooperative
 * launch) on `stream`; each arrives once and waits for nctas + missing
 * arrivals, at most wait_ns nanoseconds (0..1e9).  missing = 0: the wait
 * completes; missing > 0: it can only run out, every CTA records
 * MP_ETIMEOUT in the device error word and returns (the GPU and the
 * context stay usable), which mp_check_device_status then reports.
 * Errors: MP_EINVAL (sizes), MP_ECUDA.                                  */
int mp_grid_wait_test(int32_t nctas, int64_t wait_ns, int32_t missing, void *stream);
/* Diagnostic of the FP64 helpers of the native flux kernels (res_calc,
 * Sec. 3.1.1, and its adjoint); not in the paper.  For n doubles, mode 0:
 * y = 1/x and mode 1: y = 1/(2 x), by one third-order Newton-Raphson step
 * from an FP32 seed (the IEEE quotient for x whose exponent field is
 * outside [1, 2040]); mode 2: y = x/2 by an exponent decrement (exact; x *
 * 0.5 where that is not exact).  x and y are device arrays of n doubles
 * owned by the caller; asynchronous on `stream`.  Errors: MP_EINVAL (n < 0,
 * a null or host array with n > 0, mode not 0..2), MP_ECUDA.            */
int mp_recip_test(const double *x, double *y, int64_t n, int32_t mode, void *stream);
/* Library version string. */
const char *mp_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MESHLOOP_H */

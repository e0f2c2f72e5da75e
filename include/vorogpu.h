/*
 * vorogpu.h -- C ABI of the GB300 library for the cell-based Voronoi method
 * of "An extension to Voro++ for multithreaded computation of Voronoi cells"
 * (arXiv 2209.11606).
 *
 * The library computes, for every particle, its Voronoi cell (or radical
 * Voronoi cell) inside a rectangular container, and reduces per-cell
 * statistics.  The method is the paper's Sec. 2.1:
 *   - particles are sorted into a grid of equal blocks (Sec. 2.1.1);
 *   - a cell starts as the container box relative to its particle
 *     (Eqs. 1-2) and is cut by the half-space of Eq. 3 for each neighbour,
 *     visited near-to-far, until the radius bound of Sec. 2.1.3 shows that
 *     no remaining particle can cut it;
 *   - statistics are taken from the finished cell (Sec. 2.1.2).
 *
 * Conventions for every call:
 *   - Every function returns a vg_status; nothing throws across the ABI.
 *     On failure vg_last_error() gives a one-line reason.
 *   - The caller owns every input and output buffer it passes; the context
 *     owns its internal device buffers and frees them in vg_destroy().
 *   - `on_device` = 1 means the pointer is CUDA device memory (for example a
 *     torch tensor's data_ptr()); 0 means host memory.  Host outputs are
 *     written synchronously; device outputs are written asynchronously on
 *     the context's stream.
 *   - All work is queued on the CUDA stream given to vg_create() (NULL =
 *     the legacy default stream); the caller synchronises that stream.
 *   - A context is not thread-safe; use one context per host thread.
 *   - Cells are reported in the caller's original particle order.
 *   - Particle count is limited to 2^31 - 1 (neighbour ids are int32); the
 *     sorted-candidate prefetch form is used up to 2^27 particles and the
 *     plain walk beyond.
 */
#ifndef VOROGPU_H
#define VOROGPU_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vg_ctx vg_ctx;

typedef enum {
    VG_OK = 0,
    VG_ERR_ARG = 1,        /* invalid argument (NULL, size, dimension) */
    VG_ERR_OOM = 2,        /* device allocation failed */
    VG_ERR_OUT_OF_BOX = 3, /* a walled coordinate lies outside [lo, hi] */
    VG_ERR_NONFINITE = 4,  /* a coordinate or radius is NaN or infinite */
    VG_ERR_CAP = 5,        /* some cell exceeded every capacity tier */
    VG_ERR_CUDA = 6,       /* a CUDA call failed; see vg_last_error() */
    VG_ERR_STATE = 7,      /* call out of order (e.g. compute before insert) */
    VG_ERR_DUP_POINT = 8   /* two particles coincide (undefined bisector) */
} vg_status;

/* Arithmetic forms of the cell computation. */
enum {
    VG_FP64 = 0,        /* plain form: every cut and statistic in FP64 */
    VG_FP32_RETEST = 1  /* FP32 cuts relative to the particle; any vertex
                           within the FP32 band of a cutting plane is
                           re-tested in FP64 from the original positions;
                           volumes accumulated in FP64 */
};

/* Order in which neighbours are offered to a cell. */
enum {
    VG_WALK = 0,     /* Sec. 2.1.3: own block, then blocks in order of their
                        distance bound, stopped by the radius bound */
    VG_PREFETCH = 1  /* the candidates of the 27 surrounding blocks within a
                        prefetch radius, sorted by distance and cut in that
                        order; the radius bound still decides, and a cell
                        that needs more falls back to VG_WALK */
};

/* Per-cell status values written by vg_get_cells(). */
enum {
    VG_CELL_OK = 0,
    VG_CELL_EMPTY = 1,   /* radical variant: the cell does not exist
                            (Sec. 2.2.3: compute_cell returns false) */
    VG_CELL_CAP = 2,     /* on every tier: vertex or face capacity exceeded,
                            or a numerical failure (a new vertex off its old
                            edge or not finite, a Voronoi cell with no vertex
                            left, an inconsistent face walk) */
    VG_CELL_DUP = 3,     /* another particle sits on this one */
    VG_CELL_LIMIT = 4    /* the walk ran past its shell limit */
};

typedef struct {
    int precision;     /* VG_FP64 or VG_FP32_RETEST */
    int order;         /* VG_WALK or VG_PREFETCH */
    double tol32;      /* FP32 band: |d| <= tol32 * R * |q| is re-tested in
                          FP64 (R: current max vertex distance); default 1e-5 */
    double tau_rel;    /* FP64 on-plane band: |d| <= tau_rel * s * |q| counts
                          as on the plane and the vertex stays (s = mean
                          spacing (V/N)^(1/dim)); default 1e-11 */
    double merge_rel;  /* vertices closer than merge_rel * s are one vertex
                          (degree > 3 on exact lattices); default 1e-9 */
    int prefetch_k;    /* VG_PREFETCH: target candidate count; <= 0: the
                          library default (3D 72, 2D 24) */
    int use_mlp;       /* VG_PREFETCH: 1 = take the per-block candidate count
                          written by vg_mlp_predict() after the last insert */
    int chunk;         /* cells taken per work-queue ticket; <= 0: default */
    int warps_per_cta; /* 3D cells per CTA (one warp each), 1..4; <= 0: 4 */
    int collect_stats; /* 1 = fill the per-cell work counters */
    int time_kernels;  /* 1 = record CUDA events around the cell kernels on the
                          context's stream (read with vg_get_kernel_ms) */
    double clip;       /* clipped cells (Sec. 3.1.3): > 0 starts every cell
                          from the box intersected with the cube (2D: square)
                          of side `clip` centred on its particle; the cube's
                          faces are reported as walls (ids -1..-6 by axis and
                          side).  0 (default): plain cells */
    int weinberg;      /* 1 = also the Weinberg code of every 3D cell's edge
                          graph (Sec. 4), read with vg_get_weinberg(); either
                          form, vg_compute or a captured graph.  Default 0 */
    int split;         /* FP32 form.  3D prefetch, 1 (default): a kernel built
                          for the common path alone computes every cell it
                          can, and hands each cell that needs the walk after
                          its preloads, FP64 statistics, more than 64 planes
                          or more than 32 faces to the general kernel, which
                          computes that cell from the start (vg_get_deferred
                          counts them).  2D, 1: the first kernel holds 16
                          vertices a cell and hands larger cells to one of 32
                          (0: 32 from the start).
                          3D, 0: the general kernel computes every cell.
                          0 is better where many cells outgrow their preload
                          or 16 vertices, as in clustered sets.  The cells
                          are the same (values to rounding) */
} vg_config;

/* Fills `cfg` (caller-owned) with the defaults listed above (FP32_RETEST,
 * PREFETCH); the arithmetic forms, orders and options are this library's
 * (the paper computes in FP64 with the block walk of Sec. 2.1.3).  No error
 * (a NULL cfg is ignored). */
void vg_config_default(vg_config *cfg);

/*
 * Creates a container: the box [lo, hi] (dim = 2 or 3 doubles each), the
 * periodic flag per axis (Sec. 2.1.1), and the block grid.  `nblocks` gives
 * blocks per axis; NULL selects the Sec. 2.1.4 rule from `n_opt` particles
 * per block at the time of vg_insert() (lambda = (N/(n_opt V))^(1/dim),
 * n_a = max(1, floor(lambda L_a)); n_opt <= 0 selects 4.6 in 3D, 3.4 in 2D).
 * `stream` is a cudaStream_t (NULL: default stream).
 */
vg_status vg_create(vg_ctx **out, int dim, const double *lo, const double *hi,
                    const int *periodic, const int *nblocks, double n_opt,
                    void *stream);

/*
 * One particle system of a batched container: its box, periodic flags and
 * block grid exactly as the arguments of vg_create() (nblocks all > 0: fixed
 * counts; any <= 0: the n_opt rule at insert time).  Unused axes (dim = 2:
 * index 2) are ignored.
 */
typedef struct {
    double lo[3], hi[3];
    int periodic[3];
    int nblocks[3];
    double n_opt;
} vg_system;

/*
 * Creates a container of `nsys` independent systems that are sorted and
 * computed together: one counting sort over all of them (the system's first
 * block is added to every block key) and one persistent cell launch that
 * takes cells of all systems from one work queue -- the GPU form of the
 * paper's dynamic schedule over cells (Sec. 2.2.4), extended across systems.
 * A system's cells see only its own particles.  `systems` is read during the
 * call (caller-owned).  Errors: VG_ERR_ARG for dim not 2/3, nsys < 1, an
 * empty box or a block count above 2^20.
 */
vg_status vg_batch_create(vg_ctx **out, int dim, int nsys, const vg_system *systems,
                          void *stream);

/*
 * Replaces the particles of every system of a batched container.  counts[k]
 * (nsys entries) particles belong to system k; `pos` holds all systems' rows
 * one system after another (sum(counts) x dim values of type `dtype`) and
 * `radii` (or NULL) likewise.  Cell i and neighbour ids use this
 * concatenated numbering, so system k's cells are the input indices
 * [sum(counts[<k]), sum(counts[<=k])).  Validation and errors as
 * vg_insert() (the paper's clear() and add_parallel(), Sec. 2.2.5, for every
 * system); the per-system n_opt rule (Sec. 2.1.4) fixes the grids here.
 */
vg_status vg_batch_insert(vg_ctx *ctx, const int64_t *counts, const void *pos,
                          const void *radii, int dtype, int on_device);

/* Element type of the input positions and radii. */
enum {
    VG_F64 = 0,  /* double */
    VG_F32 = 1   /* float: widened to double on the device before the sort,
                    so the cells are those of the FP32 values read as FP64 */
};

/*
 * Replaces the container's particles (the paper's clear() followed by
 * add_parallel(), Sec. 2.2.5) and sorts them into blocks with a counting
 * sort on the GPU.  `pos` is n x dim values, row-major, and `radii` n values
 * or NULL (NULL: plain Voronoi; non-NULL: radical variant), both of type
 * `dtype` (VG_F64 or VG_F32; VG_ERR_ARG otherwise).  Coordinates on a
 * periodic axis are wrapped into [lo, hi); on a walled axis they must lie
 * in [lo, hi] (VG_ERR_OUT_OF_BOX otherwise; a point on hi goes to the last
 * block).  A NaN or infinite coordinate, or a radius that is negative or
 * not finite, gives VG_ERR_NONFINITE.  Inside a block particles are ordered
 * by input index, so results do not depend on thread timing.
 */
vg_status vg_insert(vg_ctx *ctx, int64_t n, const void *pos, const void *radii, int dtype,
                    int on_device);

/*
 * Computes every cell of the inserted particles with the given configuration
 * (`cfg` read during the call; NULL: defaults): the container box relative
 * to the particle (Eqs. 1-2) cut by the half-space of Eq. 3 for each
 * neighbour, visited near to far until the radius bound of Sec. 2.1.3
 * ends the search, then the statistics of Sec. 2.1.2.  Results stay in the
 * context until the next compute or insert (read with the vg_get_* calls).
 * Errors: VG_ERR_STATE before an insert, VG_ERR_ARG for an invalid
 * configuration (see vg_config), VG_ERR_OOM when a device buffer cannot
 * grow, VG_ERR_CAP when the face buffer still overflows after growing three
 * times, VG_ERR_CUDA on another CUDA failure.  A cell that exceeds every
 * capacity tier is reported VG_CELL_CAP in its status, not as an error.
 */
vg_status vg_compute(vg_ctx *ctx, const vg_config *cfg);

/*
 * Computes only the cells of the m input indices in `cells` (host or device
 * int32 per on_device, caller-owned), e.g. a sample for timing a
 * configuration (the method of vg_compute(); the paper's cells are
 * independent, Sec. 2.2, so a subset is computed the same way).  The
 * per-cell arrays of the listed cells then equal those of vg_compute();
 * those of other cells are unspecified, and vg_get_faces / vg_get_counts
 * return VG_ERR_STATE until the next full compute.  VG_ERR_ARG for an index
 * outside [0, n).
 */
vg_status vg_compute_subset(vg_ctx *ctx, const vg_config *cfg, const int32_t *cells, int64_t m,
                            int on_device);

/*
 * CUDA graph of one whole step (the paper has no counterpart; it replaces
 * the per-step host work of vg_insert + vg_compute).  Captures, into a graph
 * owned by the context: the counting sort of counts[k] particles of system k
 * (one entry per system; one for a vg_create container) read from the DEVICE
 * arrays `pos` (n x dim values) and `radii` (n values or NULL) of type
 * `dtype` (VG_F64 or VG_F32, as vg_insert()), the cell kernels with `cfg`
 * (NULL: defaults) and the face compaction.  Before
 * capturing it runs one eager vg_insert + vg_compute on the same input: that
 * validates the input, sizes every buffer (the face buffer with 25 %
 * headroom) and leaves valid results.  The caller keeps `pos` and `radii` at
 * the same addresses while the graph exists and may overwrite their contents
 * between replays (same counts).  Any later vg_insert, vg_batch_insert or
 * vg_compute drops the graph.  With cfg->time_kernels = 1 every replay
 * records the cell-kernel time read by vg_get_kernel_ms() and the sort time
 * read by vg_get_sort_ms().
 * Errors: VG_ERR_ARG (host input pointers, bad counts), those of vg_insert()
 * and vg_compute(), VG_ERR_CUDA when capture or instantiation fails.
 */
vg_status vg_graph_capture(vg_ctx *ctx, const int64_t *counts, const void *pos,
                           const void *radii, int dtype, const vg_config *cfg);

/* Replays the captured graph (the step of vg_graph_capture(): Sec. 2.1.1
 * sort, Sec. 2.1.3 cells, Sec. 2.1.2 statistics) on the context's stream;
 * asynchronous, input errors are read by vg_graph_sync().  VG_ERR_STATE
 * when no graph is held, VG_ERR_CUDA when the launch fails. */
vg_status vg_graph_launch(vg_ctx *ctx);

/*
 * Waits for the last replay and reads its flags: VG_ERR_OUT_OF_BOX or
 * VG_ERR_NONFINITE as vg_insert() (Sec. 2.2.5) reports them; if the replay's input made
 * more faces than the face buffer holds, the step is redone eagerly with a
 * larger buffer and the graph re-captured (VG_OK, results complete).  The
 * vg_get_* calls do this themselves after a replay.
 */
vg_status vg_graph_sync(vg_ctx *ctx);

/* Number of cells and total number of faces (edges in 2D; the face list of
 * Sec. 2.1.2) of the last vg_compute(), written to the caller's host
 * variables (either may be NULL); synchronises the stream.  VG_ERR_STATE
 * before a compute or after vg_compute_subset(). */
vg_status vg_get_counts(vg_ctx *ctx, int64_t *n_cells, int64_t *n_faces);

/*
 * Per-cell statistics of Sec. 2.1.2, n entries each, in input order, into
 * caller-owned buffers (any pointer may be NULL to skip it); VG_ERR_STATE
 * before a compute:
 *   vol       volume (3D) or area (2D), FP64
 *   area      total face area (3D) or perimeter (2D), FP64
 *   centroid  n x dim, relative to the particle, FP64
 *   nv ne nf  vertex, edge and face counts (2D: nv = ne = nf = edges)
 *   status    VG_CELL_* code
 */
vg_status vg_get_cells(vg_ctx *ctx, double *vol, double *area, double *centroid,
                       int32_t *nv, int32_t *ne, int32_t *nf, uint8_t *status,
                       int on_device);

/*
 * The neighbour list and face orders of Sec. 2.1.2, as a CSR in
 * caller-owned buffers sized by vg_get_counts() (VG_ERR_STATE before a full
 * compute): face_off has n+1 entries; cell i's faces are
 * [face_off[i], face_off[i+1]) in canonical order, ascending (neighbour id,
 * image shift).  nbr_id is the neighbour's input index, or -1..-6 for the
 * walls x-, x+, y-, y+, z-, z+ of a walled axis; nbr_img is the periodic
 * image shift of the neighbour, 3 int8 per face (z = 0 in 2D); face_order is
 * the number of vertices of the face (2 in 2D).
 */
vg_status vg_get_faces(vg_ctx *ctx, int64_t *face_off, int32_t *nbr_id, int8_t *nbr_img,
                       uint8_t *face_order, int on_device);

/*
 * Per-cell work counters of the last vg_compute() with collect_stats = 1
 * (the work of Eq. 3's cuts and of the search of Sec. 2.1.3), n entries
 * each into caller-owned buffers (any may be NULL; VG_ERR_STATE before a
 * compute): candidates offered to the cut routine,
 * vertex-plane tests, cuts that removed something, vertices those cuts
 * created, FP64 re-tests, how the prefetch form met a shortfall of its
 * preload (0 none, 1 the walk, 2 a second, wider preload), and how many
 * candidates the prefetch preloaded (both preloads; 0 for the walk).
 */
vg_status vg_get_work(vg_ctx *ctx, int32_t *n_tested, int32_t *n_vtests, int32_t *n_cuts,
                      int32_t *n_newv, int32_t *n_retest, uint8_t *fallback, int32_t *n_prefetch,
                      int on_device);

/*
 * R of every cell of the last vg_compute(): its largest vertex distance from
 * the particle (FP32; 0 for empty or failed cells), the radius whose double
 * bounds the neighbour search (Sec. 2.1.3).  n floats, input order.
 */
vg_status vg_get_radius(vg_ctx *ctx, float *rmax, int on_device);

/*
 * Weinberg codes (Sec. 4) from the last vg_compute() or graph replay with
 * cfg.weinberg = 1,
 * per cell in input order (n entries each, host or device memory):
 *   len  darts traversed, 2E (E edges of the cell's edge graph, coincident
 *        vertices merged: on an exact lattice four or more faces meet at
 *        a vertex); 0 = no code: the cell is not OK or has more than 64
 *        vertices before merging (a larger capacity tier)
 *   hash FNV-1a 64 over the 2E+1 vertex labels of the minimal code (order of
 *        first visit from 1, each label as two little-endian bytes); two
 *        cells are topologically equal iff their codes are, so equal
 *        hashes mark equal cells
 *   sym  the number of (start dart, rotation direction) pairs that give the
 *        minimal code: the order of the cell's combinatorial symmetry group
 *        (mirror images included)
 * The code traverses the edge graph from a start dart; at a new vertex it
 * leaves by the next dart after the reverse of the arriving one, at an old
 * vertex it returns along that reverse if untraversed, else leaves by the
 * first untraversed dart after it; labels list the start and every arrival.
 * The cell's code is the lexicographic minimum over all start darts and
 * both rotation directions.  VG_ERR_STATE without such a compute.
 */
vg_status vg_get_weinberg(vg_ctx *ctx, int32_t *len, uint64_t *hash, int32_t *sym, int on_device);

/*
 * Device time of the cell-kernel phase (the cuts and statistics of Sec.
 * 2.1.2-2.1.3) of every vg_compute() or graph replay made with
 * time_kernels = 1 since the previous call of this function: the sum in
 * milliseconds and the number of computes, into the caller's host
 * variables.  Synchronises the stream.  VG_ERR_ARG for NULL outputs.
 */
vg_status vg_get_kernel_ms(vg_ctx *ctx, double *total_ms, int64_t *count);

/*
 * Device time of the counting sort (FP32 widening, largest radius, block
 * keys and slots, scans, scatter, in-block order, learned preload targets:
 * Sec. 2.1.1 and Sec. 2.2.5) in every graph replay captured with
 * time_kernels = 1 since the previous call of this function: the sum in
 * milliseconds and the number of replays.  Synchronises the stream.
 */
vg_status vg_get_sort_ms(vg_ctx *ctx, double *total_ms, int64_t *count);

/*
 * Diagnostics of the cell phase (Sec. 2.1.3) in the 3D FP32 prefetch form
 * with vg_config.split = 1, into the caller's host variable: the
 * number of cells that the last vg_compute() or graph replay handed from
 * the kernel built for the common path to the general kernel (the walk
 * after both preloads, FP64 statistics, plane slots used up, more than 32
 * faces); 0 for every other form.  Synchronises the stream.
 * VG_ERR_STATE before the first compute.
 */
vg_status vg_get_deferred(vg_ctx *ctx, int64_t *count);

/*
 * Batched 3D containers (the work queue of Sec. 2.2.4 across systems), FP32
 * prefetch form with vg_config.split = 1: which kernel computes the cells of
 * system k.  split = 1 (the default for every
 * system): the kernel built for the common path, as for a single system;
 * 0: the general kernel computes all of the system's cells (better for
 * systems whose cells outgrow their preload, as clustered ones; the
 * autotuner chooses per distribution class).  Kept until changed, also in
 * a captured graph.  The cells are the same either way.  Synchronises the
 * context's stream.  VG_ERR_ARG for k out of range or split not 0 or 1.
 */
vg_status vg_set_system_split(vg_ctx *ctx, int k, int split);

/*
 * The sorted container of Sec. 2.1.1 (the blocks' particle lists):
 * block_start has B+1 entries (B = product of the block counts; for a
 * batched container the sum over systems, system k's blocks following those
 * of systems < k) and order[k] is the input index of the k-th particle in
 * block order; *n_blocks receives B.  For checking the counting sort;
 * caller-owned device or host outputs.  VG_ERR_STATE before an insert.
 */
vg_status vg_get_sorted(vg_ctx *ctx, int64_t *n_blocks, int32_t *block_start, int32_t *order,
                        int on_device);

/* Number of CUDA kernels this context has launched since vg_create()
 * (diagnostics of this library, no counterpart in the paper: lets a caller
 * count the GPU work behind a call).  VG_ERR_ARG for a NULL output. */
vg_status vg_get_launches(vg_ctx *ctx, int64_t *count);

/* The block counts in use (the grid of Sec. 2.1.1, sized by the Sec. 2.1.4
 * rule after vg_insert() when n_opt applies), dim ints into the caller's
 * host array; for a batched container, those of system 0.  VG_ERR_ARG for
 * a NULL output. */
vg_status vg_get_grid(vg_ctx *ctx, int *nblocks);

/* The block counts (Sec. 2.1.1) of system k of a (batched) container, as
 * vg_get_grid().  VG_ERR_ARG for k out of range. */
vg_status vg_get_system_grid(vg_ctx *ctx, int k, int *nblocks);

/* ---- learned candidate count ---------------------------------------------
 *
 * The paper has no learned part; its cells take candidates from the block
 * walk with the radius bound (Sec. 2.1.3).  The prefetch form of the cell
 * kernel preloads, in one batch, the candidates in a ball expected to hold k
 * of them (k from the local density of the 27 surrounding blocks), sorts them
 * by distance and cuts them in order; the radius bound still decides and a
 * shortfall falls back to the walk, so cells never depend on k.  These calls
 * train and run a small network that predicts k per block from the 27 block
 * counts:
 *
 *   features  x_j = c_j / m - 1, c_j the count of block b + (dx,dy,dz),
 *             j = (dx+1) + 3 (dy+1) + 9 (dz+1), wrapped on periodic axes,
 *             0 past a wall, m the mean count of those of the 27 blocks
 *             inside the box (x = 0 where m = 0): counts relative to their
 *             local mean, the same at any density or block size;
 *   network   y = W3 . relu(W2 relu(W1 x + b1) + b2) + b3, hidden widths 32
 *             and 32, W1 W2 W3 in FP16, biases FP32, FP32 accumulation;
 *             predicted count exp(y);
 *   label     k*_i = candidates (particle, periodic image) within 2 R_i of
 *             cell i (R_i from vg_get_radius), the particle itself excluded;
 *   target    t_b = log(max(1, max k* over block b's cells));
 *   loss      (1/M) sum_b w_b (y_b - t_b)^2, w_b = u if y_b < t_b else 1;
 *   update    Adam, beta1 0.9, beta2 0.999, eps 1e-8, on FP32 master
 *             weights; the FP16 copy is refreshed after every step.
 *
 * Parameters are 1985 floats packed as W1 (32 x 27, row per hidden unit),
 * b1 (32), W2 (32 x 32), b2 (32), W3 (32), b3 (1).
 */
typedef struct vg_mlp vg_mlp;

/* A predictor (the learned count above) with all parameters 0, owned by
 * the caller until vg_mlp_destroy(); its work goes on `stream`.  VG_ERR_ARG
 * for a NULL `out`, VG_ERR_OOM when its buffers cannot be allocated,
 * VG_ERR_CUDA on another CUDA failure. */
vg_status vg_mlp_create(vg_mlp **out, void *stream);
void vg_mlp_destroy(vg_mlp *mlp);
const char *vg_mlp_last_error(vg_mlp *mlp);

/* Sets the FP32 master parameters of the network above (1985 host floats,
 * read during the call), refreshes the FP16 copy and clears the Adam state.
 * VG_ERR_ARG for NULL. */
vg_status vg_mlp_set_params(vg_mlp *mlp, const float *params);
/* Copies the FP32 master parameters of the network above to 1985
 * caller-owned host floats.  VG_ERR_ARG for NULL. */
vg_status vg_mlp_get_params(vg_mlp *mlp, float *params);

/* Features (above) of every block of an inserted container (all systems,
 * global block order): total blocks x 27 floats, row-major, caller-owned.
 * VG_ERR_STATE before an insert, VG_ERR_ARG for a NULL output. */
vg_status vg_mlp_features(vg_ctx *ctx, float *X, int on_device);

/* k* (above: candidates within twice the cell's radius, the bound of
 * Sec. 2.1.3) of every cell of the last vg_compute() (n int32, input order,
 * caller-owned).  VG_ERR_STATE before a compute. */
vg_status vg_mlp_labels(vg_ctx *ctx, int32_t *kstar, int on_device);

/*
 * Training rows (features and targets above) from the last vg_compute():
 * one per block holding a particle, in block order: features into X
 * (DEVICE, caller-owned, room for total blocks x 27 floats) and targets into
 * t (DEVICE, room for total blocks floats); *m receives the number of rows.
 * VG_ERR_ARG for NULL outputs, VG_ERR_STATE before a compute.
 */
vg_status vg_mlp_dataset(vg_ctx *ctx, float *X, float *t, int64_t *m);

/* Loss and gradient (above) over M device rows (X: M x 27, t: M,
 * caller-owned) at the current FP16 weights, without an update; grad is
 * 1985 host floats (may be NULL).  VG_ERR_ARG for M < 1 or NULL rows. */
vg_status vg_mlp_loss_grad(vg_mlp *mlp, const float *X, const float *t, int64_t M, float u,
                           double *loss, float *grad);

/* `steps` full-batch Adam steps (above) over M device rows with learning
 * rate lr and under-prediction weight u; losses (host, `steps` floats, may
 * be NULL) receives the loss before each step.  VG_ERR_ARG for M < 1,
 * steps < 0, lr <= 0 or NULL rows. */
vg_status vg_mlp_train(vg_mlp *mlp, const float *X, const float *t, int64_t M, float u, float lr,
                       int steps, float *losses);

/* Network output y (above) for M device rows of features (y: M device
 * floats, caller-owned).  VG_ERR_ARG for M < 0 or, with M > 0, NULL
 * buffers. */
vg_status vg_mlp_infer(vg_mlp *mlp, const float *X, int64_t M, float *y);

/*
 * Per-block preload targets (the learned count above) for the inserted
 * container: clamp(alpha exp(y),
 * kmin, kmax) for every block, used by vg_compute() with use_mlp = 1 until
 * the next insert (each block preloads the geometric mean of the targets
 * of its 27 blocks, at least 8).  VG_ERR_STATE before an insert.
 */
vg_status vg_mlp_predict(vg_ctx *ctx, vg_mlp *mlp, float alpha, float kmin, float kmax);

/*
 * Attaches a predictor to a container (NULL detaches): every later sort
 * (vg_insert, vg_batch_insert, graph replays) is followed by the prediction
 * of vg_mlp_predict(), so use_mlp = 1 needs no separate call and a captured
 * graph runs sort -> predict -> cells -> faces (the preload target of the
 * prefetch form; the search of Sec. 2.1.3 still decides).  The container
 * does not own the predictor, which must outlive its use; attach again
 * after training it further.  VG_ERR_ARG for a NULL context or, with a
 * predictor, alpha <= 0, kmin <= 0 or kmax < kmin.
 */
vg_status vg_set_predictor(vg_ctx *ctx, vg_mlp *mlp, float alpha, float kmin, float kmax);

/*
 * Counting sort into blocks that allocates no device memory.  The paper has
 * no counterpart: it is a variant of the sort inside vg_insert() for callers
 * that must not allocate at call time -- for example a plugin whose host
 * framework owns all device memory and forbids allocation on its execution
 * path, a latency-critical loop that cannot absorb the device
 * synchronisation cudaMalloc/cudaFree imply, or a process near its memory
 * limit.  The sort's scratch (keys, slots, block counts) lives in one fixed
 * __device__ array inside the library, about 13 MB, which every device that
 * loads the library holds until the process exits.
 *
 *   dim, lo, hi, periodic, nblocks   the container, as in vg_create()
 *   n, pos      n x dim doubles in DEVICE memory; n <= 1,048,576
 *   block_start DEVICE output, B + 1 int32 (B = product of nblocks <= 262,144)
 *   order       DEVICE output, n int32: input index of each particle in block
 *               order, ascending input index inside a block -- the same
 *               arrays vg_get_sorted() returns after vg_insert()
 *   stream      cudaStream_t (NULL: default stream); the call synchronises it
 *   errbuf      optional caller buffer of errlen bytes for a one-line reason
 *
 * Returns VG_ERR_ARG (with the reason in errbuf) when n or B exceeds the
 * limits above, VG_ERR_OUT_OF_BOX / VG_ERR_NONFINITE as vg_insert() does,
 * VG_ERR_CUDA on a CUDA failure.  It calls no cudaMalloc, cudaFree or other
 * allocating routine.  Every call ends by reading the error flags back to a
 * host variable and synchronising `stream`.  The first call on each device
 * looks up the device address of the scratch array (cudaGetSymbolAddress)
 * with that device current and keeps it for the rest of the process; do
 * not call this entry point after resetting the device (cudaDeviceReset),
 * which would leave the kept address stale.  All calls on a device share the one scratch array,
 * so calls that overlap on the GPU (from two streams or two host threads)
 * race and must be serialised by the caller.
 */
vg_status vg_sort_blocks_noalloc(int dim, const double *lo, const double *hi, const int *periodic,
                                 const int *nblocks, int64_t n, const double *pos,
                                 int32_t *block_start, int32_t *order, void *stream,
                                 char *errbuf, int errlen);

const char *vg_last_error(vg_ctx *ctx);
void vg_destroy(vg_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* VOROGPU_H */

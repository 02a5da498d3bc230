/*
 * dog.h -- C ABI of the B300-native DS-PHD/MIB dynamic occupancy grid filter.
 *
 * The filter is the Dempster-Shafer approximation of the PHD/MIB filter of Nuss et al.,
 * "A Random Finite Set Approach for Dynamic Occupancy Grid Maps with Real-Time
 * Application" (Sect. VI), computed by the parallel recursion of Sect. VII (Alg. 1-7):
 * particle prediction, sorting particles by grid cell, occupancy prediction and update,
 * normalisation of persistent particles, initialisation of newborn particles, velocity
 * moments and resampling.
 *
 * Conventions
 *   - Every call returns DOG_OK (0) or a negative dog_status; nothing throws or aborts.
 *   - The library owns no device memory: dog_create carves every array out of a device
 *     workspace the caller allocates (size from dog_workspace_bytes) and keeps alive until
 *     dog_destroy.  dog_destroy never frees it.
 *   - All device work of a filter is issued on the CUDA stream given to dog_create, in
 *     call order.  Calls marked "asynchronous" return before the GPU has finished.
 *   - A handle is not thread-safe: calls on one filter must be serialised by the caller.
 *   - Arrays are SoA; cell arrays have C = width * height entries in row-major order
 *     (cell index = row * width + col, row = floor(y / cell_size), col = floor(x / cell_size),
 *     grid origin at the corner (0, 0)).
 *   - Errors detected on the device (an input that fails validation, an internal
 *     consistency check) are latched in the filter and returned by the next synchronising call
 *     (dog_get_cells, dog_get_state, dog_get_debug, dog_sync), which clears them.  While an
 *     error is latched, the results of the frames that follow are void.
 */
#ifndef DOG_H
#define DOG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum dog_status {
  DOG_OK = 0,
  DOG_ERR_INVALID_ARG = -1,         /* bad pointer, size or parameter                   */
  DOG_ERR_WORKSPACE_TOO_SMALL = -2, /* workspace smaller than dog_workspace_bytes        */
  DOG_ERR_CUDA = -3,                /* a CUDA runtime call failed                        */
  DOG_ERR_DEVICE = -4,              /* a device-side consistency check failed; void      */
  DOG_ERR_INPUT = -5,               /* measurement grid / state outside its domain       */
  DOG_ERR_BAD_STATE = -6,           /* call not valid in the filter's current state      */
  DOG_ERR_UNSUPPORTED = -7          /* size beyond the supported maximum                 */
} dog_status;

/* dog_params.flags */
#define DOG_NO_RESAMPLE 0x2u /* keep the normalised persistent particles (test mode)     */
#define DOG_RECORD 0x4u      /* also keep newborn cells/sets and explicit cell ranges     */
#define DOG_NO_GRAPH 0x8u    /* issue kernels one by one instead of a captured graph     */
#define DOG_PROFILE 0x10u    /* time each kernel with CUDA events (dog_profile_read)      */
#define DOG_EGO 0x20u        /* the grid moves with the vehicle: dog_set_ego_motion         */
#define DOG_FULL 0x40u       /* the PHD/MIB filter of Sect. VI with its Bernoulli observation
                                (dog_set_bernoulli_grid) instead of the DS approximation */
#define DOG_AUTOTUNE 0x80u   /* reserve the buffers of a sort with one pass more, so that
                                dog_autotune / dog_set_sort_config may choose it */

/* memory kind of caller buffers */
#define DOG_HOST 0
#define DOG_DEVICE 1
#define DOG_HOST_ASYNC 2 /* dog_set_measurement_grid only: host arrays, the call does not wait */

/* Filter parameters (Table I of the paper gives typical values).  All POD; validated by
 * dog_workspace_bytes and dog_create.  Limits: 1 <= width, height; C = width*height < 2^24 (so
 * the 2^-40 fixed-point total of all cell masses, at most C, stays below 2^64);
 * 1 <= num_particles < 2^25; num_birth < 2^25. */
typedef struct dog_params {
  int32_t width, height;   /* grid cells                                             */
  float cell_size;         /* m                                                      */
  uint32_t num_particles;  /* nu, persistent particles (constant, Sect. V-F)         */
  uint32_t num_birth;      /* nu_b, newborn particles per frame (constant, Sect. VII) */
  float p_S;               /* persistence probability, Eq. particle_persistence      */
  float p_B;               /* birth probability, Eq. DS_resulting_masses1            */
  float alpha_free;        /* free-mass discount alpha(T), Eq. DS_freespace_pred     */
  float sigma_pos;         /* per-frame process noise SD of position (m), Eq. process */
  float sigma_vel;         /* per-frame process noise SD of velocity (m/s)           */
  float sigma_birth_vel;   /* SD of newborn velocities (m/s), Table I                 */
  float sensor_x, sensor_y;/* radar position (m) for the radial-velocity likelihood  */
  uint64_t seed;           /* Philox4x32-10 key                                       */
  uint32_t flags;          /* DOG_* flags above                                       */
} dog_params;

/* Measurement grid (the paper's meas_cell_array, Sect. VII), SoA with C entries each.
 * m_occ, m_free: observed occupancy BBA, each in [0,1], m_occ + m_free <= 1 (+1e-6).
 * p_A, z_vr, sigma_vr: optional (all NULL for a lidar-only grid): association
 * probability in [0,1] and the measured radial velocity with its SD (> 0 where p_A > 0)
 * of the cell's spatial likelihood (Sect. VI-C). */
typedef struct dog_meas_grid {
  const float *m_occ, *m_free;
  const float *p_A, *z_vr, *sigma_vr;
} dog_meas_grid;

/* Bernoulli observation of each cell for the PHD/MIB filter (Sect. VI, Bernoulli
 * Observation Process), SoA with C entries each: z = 1 where a measurement occurred, else 0;
 * p_tp, p_fp in (0,1): the cell's true / false positive probabilities; p_a in [0,1]: the
 * association probability; p_c > 0: the clutter density of the cell's measurement.  The
 * single-object likelihood of a measured cell is 1 over the cell (an occupancy-grid
 * detection carries no position inside the cell), so p_c is the likelihood ratio of clutter
 * to the object.  Fields of unmeasured cells other than p_tp, p_fp are not used but must
 * still lie in their ranges. */
typedef struct dog_bern_grid {
  const float *z, *p_tp, *p_fp, *p_a, *p_c;
} dog_bern_grid;

/* Per-cell outputs of the last frame; any pointer may be NULL (not copied).
 * m_occ, m_free: posterior BBA (Eq. DS_comb); rho_p, rho_b: persistent / newborn parts of
 * m_occ (Eq. DS_resulting_masses1/2); p_occ: pignistic occupancy probability (Sect. VI-A);
 * mean_vx, mean_vy, var_vx, var_vy, cov_vxy: velocity moments of the persistent
 * particles (Eq. mean_x, var_x, covar_xy), 0 where rho_p = 0. */
typedef struct dog_cells {
  float *m_occ, *m_free, *rho_p, *rho_b, *p_occ;
  float *mean_vx, *mean_vy, *var_vx, *var_vy, *cov_vxy;
} dog_cells;

/* Posterior state (checkpoint): particles x, y, vx, vy, w [num_particles] and the cells'
 * free mass m_free [C]; the frame counter travels separately. */
typedef struct dog_state {
  float *x, *y, *vx, *vy, *w;
  float *m_free;
} dog_state;

typedef struct dog_filter dog_filter; /* opaque */

/* Bytes of device workspace dog_create needs for these parameters (host arithmetic only).
 * Errors: DOG_ERR_INVALID_ARG (NULL or invalid parameters), DOG_ERR_UNSUPPORTED. */
int dog_workspace_bytes(const dog_params *params, size_t *out_bytes);

/* Create a filter in the caller's device workspace (256-byte aligned, at least
 * dog_workspace_bytes long) on cuda_stream (a cudaStream_t; NULL = legacy default stream,
 * which disables graph capture).  Initial state (frame 0): particles uniform over the grid
 * with birth-distribution velocities and weight 0; all cells m_occ = m_free = 0.
 * Asynchronous.  Errors: INVALID_ARG, UNSUPPORTED, WORKSPACE_TOO_SMALL, CUDA. */
int dog_create(const dog_params *params, void *d_workspace, size_t workspace_bytes,
               void *cuda_stream, dog_filter **out);

/* Copy a measurement grid into the filter (Sect. VII: same dimensions as the map); it is
 * used by every following dog_step until replaced.  mem_kind says where the caller's arrays
 * live.  The grid is copied and validated on the device (m_occ, m_free in [0, 1] with
 * m_occ + m_free <= 1; p_A in [0, 1]; sigma_vr > 0 where p_A > 0; z_vr finite).
 * DOG_HOST: the arrays are uploaded on the filter's upload stream (overlapping a frame
 * still in flight) and the call returns when the upload is done, so the caller may reuse
 * them; pinned host memory is fastest.  DOG_HOST_ASYNC: the same upload, but the call
 * returns at once and the caller must leave the arrays unchanged until the upload is done
 * (guaranteed after dog_sync, or after dog_get_cells_async / dog_wait_cells of a later
 * frame has returned).  DOG_DEVICE: asynchronous.  In all cases a violation
 * is latched and reported as DOG_ERR_INPUT by the next synchronising call (dog_sync,
 * dog_get_cells, dog_wait_cells, ...); the frames stepped with that grid are void. */
int dog_set_measurement_grid(dog_filter *f, const dog_meas_grid *grid, int mem_kind);

/* The same for a filter created with DOG_FULL: the PHD/MIB filter of Sect. VI.  Each frame
 * then runs the particle realisation of Sect. VI: persistent prediction as in Alg. 1;
 * r_p = min(sum of the cell's predicted weights, 1) (weights of a cell over 1 scaled to sum
 * 1); newborn existence r_b = p_B (1 - r_p) (Eq. pred_birth_prob), newborn slots shared out
 * in proportion to r_b with weights r_b / n; the Bernoulli update (Eq. filter_update with
 * normalization_empty / normalization_meas), which with a likelihood of 1 multiplies every
 * weight of the cell by f = p_tp g_A / N_z (measured, g_A = p_a + (1 - p_a) p_c, N_z =
 * p_fp p_c (1 - r) + p_tp g_A r) or f = (1 - p_tp) / ((1 - p_tp) r + (1 - p_fp)(1 - r))
 * (not measured), r = r_p + r_b; resampling as in Alg. 7.  dog_get_cells then gives
 * m_occ = p_occ = the posterior existence r' = f r (Eq. occprob_integral), m_free = 1 - r',
 * rho_p = f r_p, rho_b = f r_b.  Errors: as dog_set_measurement_grid (INPUT: z not 0 or 1,
 * a probability or p_c out of range); BAD_STATE: filter without DOG_FULL (and
 * dog_set_measurement_grid on a DOG_FULL filter). */
int dog_set_bernoulli_grid(dog_filter *f, const dog_bern_grid *grid, int mem_kind);

/* Ego-motion compensation for the next dog_step (filters created with DOG_EGO; the paper's
 * experiments compensate the vehicle's motion from speed and yaw rate, Sect. VIII, without
 * fixing how).  The grid is attached to the vehicle, the sensor at (sensor_x, sensor_y):
 * since the previous frame the vehicle moved by (dx, dy) m, in the previous grid's axes,
 * and turned by dyaw rad (counter-clockwise) about the sensor position.  At the start of
 * the next step every posterior particle enters the new grid at q + R(-dyaw)(p - q - d)
 * with velocity R(-dyaw) v (q the sensor position, d = (dx, dy)), before the process model;
 * the posterior free mass of each new cell is read at the old cell under its centre,
 * q + R(dyaw)(c - q) + d (nearest cell; 0 outside the old grid).  cos and sin of dyaw are
 * taken in binary64 and rounded to binary32 once.  Applies to one step; a step without a
 * call keeps the grid where it is.  Asynchronous (the values are passed by value).
 * Errors: INVALID_ARG (non-finite argument), BAD_STATE (filter without DOG_EGO). */
int dog_set_ego_motion(dog_filter *f, float dx, float dy, float dyaw);

/* One recursion of the filter with time step dt (s): Alg. 1-7 of Sect. VII.
 * Asynchronous.  Errors: INVALID_ARG (dt not finite or < 0), BAD_STATE (no measurement
 * grid set yet), CUDA. */
int dog_step(dog_filter *f, float dt);

/* Copy the per-cell outputs of the last frame; synchronises the filter's stream.  Returns
 * a latched device error if one occurred since the last synchronising call. */
int dog_get_cells(dog_filter *f, const dog_cells *out, int mem_kind);

/* Asynchronous read-back of the cells of the last dog_step into HOST arrays (any field NULL
 * = skipped; pinned host memory lets the copy overlap the next frame).  The requested fields
 * are copied on the device in stream order -- the next dog_step may be issued at once -- and
 * from there to the host on the filter's read-back stream.  The arrays are valid after
 * dog_wait_cells returns.  One read-back may be in flight per filter: a second call first
 * waits for the previous one.  Errors latched in stream order before the snapshot (input
 * validation of any grid set before this call) are returned by dog_wait_cells.  To keep
 * the GPU busy, upload the next frame's grid (DOG_HOST_ASYNC) before this call: dog_step(k),
 * dog_set_measurement_grid(k + 1), dog_get_cells_async(k).  Errors: INVALID_ARG, CUDA. */
int dog_get_cells_async(dog_filter *f, const dog_cells *out);

/* Block until the read-back started by dog_get_cells_async has arrived (DOG_OK at once if
 * none is in flight).  Errors: INPUT / DEVICE (latched before the read-back), CUDA. */
int dog_wait_cells(dog_filter *f);

/* Read / write the posterior state and frame counter (checkpoint / resume; Philox draws
 * depend only on (seed, frame, index), so a resumed filter continues bit-exactly).
 * dog_get_state synchronises; dog_set_state is ordered on the stream and returns after
 * its copies completed. */
int dog_get_state(dog_filter *f, const dog_state *out, int mem_kind, uint32_t *frame);
int dog_set_state(dog_filter *f, const dog_state *in, int mem_kind, uint32_t frame);

/* Sort configuration (Alg. 2: the LSD radix sort of particles by cell index): the number of
 * digit passes (the digit width is ceil(key bits / passes), at most 11) and the number of
 * sort tiles that one block of the digit-counting kernel takes (1, 2, 4 or 8).  Every
 * configuration sorts to the same order, so results are the same bit for bit; only the
 * speed differs.  The default is the fewest passes and the tiles per block that leave two
 * blocks per SM.
 *
 * dog_autotune times every configuration the workspace allows (the default number of
 * passes, and one more with DOG_AUTOTUNE) on the predicted keys of the last step, on the
 * filter's stream (it synchronises), and keeps the fastest; the choice is also cached for
 * the process by the size class (ceil log2 num_particles, ceil log2 cells) and applied to
 * filters of that class created later.  The filter's state and outputs are unchanged.  A
 * batch keeps the configuration its filters had when it was created.
 * Errors: BAD_STATE (no step yet), CUDA.
 * dog_set_sort_config sets one explicitly.  Errors: INVALID_ARG, UNSUPPORTED (a
 * configuration the workspace does not hold or an invalid tile count).
 * dog_sort_config reads the current one (any output pointer may be NULL). */
int dog_autotune(dog_filter *f);
int dog_set_sort_config(dog_filter *f, int passes, int count_tiles);
int dog_sort_config(const dog_filter *f, int *passes, int *digit_bits, int *count_tiles);

/* Wait for the filter's stream; return a latched device error, else DOG_OK. */
int dog_sync(dog_filter *f);

/* Intermediates of the last frame (for parity tests and diagnostics); synchronises.
 * which / element type / count:
 *   DOG_DBG_PRED_X..PRED_W   float [nu]  predicted particles, original order (Alg. 1)
 *   DOG_DBG_KEY              u32   [nu]  cell index of each predicted particle
 *   DOG_DBG_PERM             u32   [nu]  sorted position -> particle index (Alg. 2)
 *   DOG_DBG_CELL_START/END   u32   [C]   half-open sorted range of each cell, 0/0 if empty
 *                                  (a lidar-only filter writes them with DOG_RECORD only)
 *   DOG_DBG_SUM_W, SUM_GW    u64   [C]   fixed-point (2^-40) sums of w and g*w per cell
 *   DOG_DBG_M_OCC_PRED       float [C]   predicted occupied mass (Eq. DS_particle_sum_pred)
 *   DOG_DBG_MU_A, MU_UA      float [C]   normalisation factors (Eq. DSnormalizationfactor(2))
 *   DOG_DBG_W_NORM           float [nu]  normalised persistent weights, sorted order
 *   DOG_DBG_BIRTH_X..BIRTH_W float [nu_b] newborn particles (Alg. 5)
 *   DOG_DBG_BIRTH_CELL       u32   [nu_b] (DOG_RECORD only)
 *   DOG_DBG_BIRTH_ASSOC      u32   [nu_b] 1 = associated set (DOG_RECORD only)
 *   DOG_DBG_RESAMPLE_SRC     u32   [nu]  joint source index of each posterior particle
 *   DOG_DBG_SCALARS          u64   [4]   frame, total weight, total birth mass, offset u
 * Errors: INVALID_ARG (unknown which), BAD_STATE (needs DOG_RECORD). */
enum {
  DOG_DBG_PRED_X = 0, DOG_DBG_PRED_Y, DOG_DBG_PRED_VX, DOG_DBG_PRED_VY, DOG_DBG_PRED_W,
  DOG_DBG_KEY, DOG_DBG_PERM, DOG_DBG_CELL_START, DOG_DBG_CELL_END, DOG_DBG_SUM_W,
  DOG_DBG_SUM_GW, DOG_DBG_M_OCC_PRED, DOG_DBG_MU_A, DOG_DBG_MU_UA, DOG_DBG_W_NORM,
  DOG_DBG_BIRTH_X, DOG_DBG_BIRTH_Y, DOG_DBG_BIRTH_VX, DOG_DBG_BIRTH_VY, DOG_DBG_BIRTH_W,
  DOG_DBG_BIRTH_CELL, DOG_DBG_BIRTH_ASSOC, DOG_DBG_RESAMPLE_SRC, DOG_DBG_SCALARS,
  DOG_DBG_COUNT
};
int dog_get_debug(dog_filter *f, int which, void *out, int mem_kind);

/* Per-kernel device time (ms) summed over the steps since the last read (DOG_PROFILE,
 * which issues kernels one by one with CUDA events between them).  names[k] receives a
 * static string; *n_out the number of kernels (<= max); *steps_out the steps covered. */
int dog_profile_read(dog_filter *f, float *ms, const char **names, int max, int *n_out,
                     int *steps_out);

/* Number of kernels one dog_step launches (for launch accounting). */
int dog_kernels_per_step(const dog_filter *f);

/* Allocation-free assignment of particles to grid cells (the paper has no counterpart;
 * it is the sort-and-range step of dog_step offered to callers that cannot allocate device
 * memory -- code running where cudaMalloc is forbidden or unavailable, such as a host
 * callback, a real-time thread that must not take the allocator's locks, or a process whose
 * device memory is owned by another framework's pool).
 *   d_keys       [n] cell index of each particle (device).  A key >= num_cells (any value,
 *                including those with the top bit set) belongs to no cell: such particles
 *                are placed after all particles with valid keys, in input order, and are
 *                in no cell's range.
 *   d_perm       [n] out: stable sort permutation (sorted position -> particle index)
 *   d_cell_start, d_cell_end [num_cells] out: half-open range of each cell in sorted order,
 *                0/0 for an empty cell (the same values as DOG_DBG_PERM / CELL_START / END)
 * Limits: n <= DOG_NOALLOC_MAX_PARTICLES, 1 <= num_cells <= DOG_NOALLOC_MAX_CELLS; larger
 * sizes return DOG_ERR_UNSUPPORTED and touch nothing.  Scratch: one fixed array of
 * 10,502,400 bytes in the library's device image (held by every GPU that loads the library
 * until the process exits); no call allocates or frees memory.  Asynchronous on cuda_stream.
 * The first call in a CUDA context looks up that array's device address and sets the sort
 * kernels' shared-memory limits for the current device (make it before any stream capture);
 * later calls in the same context reuse them.  Every call on a device shares the array:
 * calls that overlap on the GPU (other streams or threads) race and must be serialised. */
#define DOG_NOALLOC_MAX_PARTICLES (1u << 19)
#define DOG_NOALLOC_MAX_CELLS ((1u << 22) - 1u)
int dog_assign_cells_noalloc(const uint32_t *d_keys, uint32_t n, uint32_t num_cells,
                             uint32_t *d_perm, uint32_t *d_cell_start, uint32_t *d_cell_end,
                             void *cuda_stream);

/* Release the handle (the caller's workspace is left untouched and may be freed after
 * the stream has drained). */
void dog_destroy(dog_filter *f);

/* ---- Batched stepping (no counterpart in the paper: a way to run many independent
 * filters per frame).  A batch advances n filters by one frame each with a single CUDA-graph
 * launch in which every phase of the frame (prediction, each sort pass, cell sums, cell
 * update, newborns, normalisation, resampling) is ONE kernel launch over the tiles of all n
 * filters: a block finds its filter and tile from a prefix table of the filters' block
 * counts, so small and large filters fill the GPU together.  Each filter's parameters and
 * buffer table are written into a 1 KB slot of its own workspace when the batch captures its
 * graph (the library still allocates no device memory).  Every filter of a batch must have
 * been created on the same non-NULL stream; the batch launches on that stream, so each
 * filter's other calls (grids, cells, state) stay ordered with the batched frames.  Filters
 * created with DOG_PROFILE cannot be batched.  A filter may belong to several batches and
 * may still be stepped alone with dog_step; the caller must not destroy a filter before the
 * batches that hold it. */
typedef struct dog_batch dog_batch;

/* Create a batch over filters[0..n) (1 <= n <= 128, distinct, pointers kept, not owned).
 * Errors: INVALID_ARG (NULL, n < 1, a filter listed twice, different or NULL streams, a
 * profiling filter), UNSUPPORTED (n > 128), CUDA. */
int dog_batch_create(dog_filter *const *filters, int n, dog_batch **out);

/* One frame of every filter of the batch, with time steps dt[0..n) (host array, s).  Each
 * filter needs a measurement grid, as for dog_step.  Asynchronous; results equal n calls of
 * dog_step bit for bit.  The graph is captured on the first call and again whenever a
 * filter's grid switched between lidar and lidar + radar, its sort configuration changed
 * (dog_autotune, dog_set_sort_config), or another batch captured it since.
 * Errors: INVALID_ARG (dt out of domain), BAD_STATE (a filter without grid), CUDA. */
int dog_batch_step(dog_batch *b, const float *dt);

/* Grouping of the batch's filters: consecutive filters (in the order given to
 * dog_batch_create) whose workspaces add up to at most group_bytes form one group; a filter
 * larger than that is a group of its own.  Each group is one branch of the batch graph, the
 * branches run concurrently, and within a group of several filters every phase of the frame
 * is one launch over all of them; a group of one filter runs its own kernels.  0 (the
 * default) makes every filter its own branch; SIZE_MAX fuses the whole batch into one group.
 * Results do not depend on the grouping.  The graph is captured again at the next step.
 * dog_batch_groups returns the current number of groups.  Errors: INVALID_ARG. */
int dog_batch_set_group_bytes(dog_batch *b, size_t group_bytes);
int dog_batch_groups(const dog_batch *b, int *n_groups);

/* Pick the grouping by measurement: steps the batch with each candidate grouping (one
 * filter per branch, groups of up to 64 MB, 256 MB, 1 GB, 4 GB of workspace, the whole batch
 * fused), `frames` timed frames each after one that captures the graph, with time steps
 * dt[0..n), and keeps the fastest (written to *chosen if not NULL).  These are real frames of
 * every filter (each needs its measurement grid, as for dog_batch_step): the filters advance
 * by one frame per step taken, results being the same under every grouping.  Synchronises
 * the batch's stream.  Errors: as dog_batch_step; INVALID_ARG (frames < 1). */
int dog_batch_autotune(dog_batch *b, const float *dt, int frames, size_t *chosen);

/* Release the batch (waits for its stream); the filters stay. */
void dog_batch_destroy(dog_batch *b);

/* ---- Evaluation against ground truth (the experiments of Sect. VIII).  Both calls read
 * the filter's current cell estimates (those of the last dog_step), take device pointers,
 * run asynchronously on the filter's stream and return DOG_ERR_INVALID_ARG for NULL or
 * empty arguments.
 *
 * dog_eval_clusters: velocity statistics of cell clusters S, one per object.
 *   d_cell_object [C] int32: 0 = no object, k = 1..n_objects the object the cell belongs to.
 *   d_scratch [n_objects][5] int64: work space (zeroed by the call).
 *   d_stats   [n_objects][5] double out: |S|; the cluster mean velocity (Eq. mean_cluster:
 *             the average of the cells' mean vx, vy); the cluster variance (Eq.
 *             gaussian_mixture_x: average of var + mean^2 minus the squared cluster mean),
 *             x then y.  Sums are exact in 2^-32 fixed point of the binary64 cell terms.
 *   The normalised estimation error squared of Eq. NEES_x follows from d_stats and the
 *   object's true velocity. */
int dog_eval_clusters(dog_filter *f, const int32_t *d_cell_object, uint32_t n_objects,
                      long long *d_scratch, double *d_stats);

/* dog_eval_mahalanobis: the Mahalanobis distance m = v P^-1 v^T of each cell's velocity
 * estimate (mean v, covariance P from var_vx, var_vy, cov_vxy) from v = 0 (Eq. mahadist;
 * binary32, 0 for a singular P with v = 0, +inf for a singular P otherwise), and a
 * classification histogram: over the cells with label 1 (dynamic) or 2 (static) and
 * m_occ >= min_occ, d_counts[(label - 1) * (n_thresholds + 1) + j] counts the cells for
 * which exactly j of the ascending d_thresholds are <= m (zeroed by the call).  A cell is
 * detected as dynamic at threshold t_j when m >= t_j, so the detections at t_j are the
 * cells counted in bins j + 1 .. n_thresholds.  d_m (optional, [C] float) receives m
 * (0 for cells not evaluated).  Errors: INVALID_ARG, UNSUPPORTED (n_thresholds > 4096). */
int dog_eval_mahalanobis(dog_filter *f, const uint8_t *d_label, float min_occ,
                         const float *d_thresholds, uint32_t n_thresholds,
                         unsigned long long *d_counts, float *d_m);

/* Static description of a dog_status. */
const char *dog_error_string(int code);

/* The CUDA runtime's description of the last CUDA failure that made a call of this thread
 * return DOG_ERR_CUDA ("" if none); static storage. */
const char *dog_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif /* DOG_H */

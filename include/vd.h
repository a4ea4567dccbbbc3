/*
 * vd.h -- C ABI of the GB300 (sm_103a) dynamic Voronoi diagram library.
 *
 * The library computes discrete 2D Voronoi diagrams (a nearest-seed index per
 * pixel) with the Jump Flooding Algorithm (JFA) and with the dynamic JFA
 * (dJFA) of "GPU Voronoi Diagrams for Random Moving Seeds" (Stevenson-Regla
 * and Navarro), every step of which runs in this library's own CUDA kernels.
 *
 * Conventions for every call below:
 *   - Coordinates and sizes are int32.  A grid is w columns by h rows,
 *     1 <= w, h <= VD_MAX_SIDE; pixel (x, y) of a dense caller map is element
 *     y * w + x (row-major, no padding).
 *   - Seeds are int32 (x, y) pairs, seed k at xy[2k], xy[2k + 1], with
 *     0 <= x < w and 0 <= y < h.  Seed indices are the labels.
 *   - Label -1 means "no seed".  Distances are exact integers: squared
 *     Euclidean (VD_METRIC_EUCLID) or Manhattan (VD_METRIC_MANHATTAN); among
 *     equal distances the lowest seed index wins, so every result is unique
 *     and bit-reproducible.
 *   - A pointer flagged `on_device` is a CUDA device pointer of the current
 *     device; otherwise it is host memory.  The caller keeps ownership of
 *     every buffer it passes; the library copies what it needs.  Host sources
 *     follow cudaMemcpyAsync rules: pageable memory may be reused when the
 *     call returns, page-locked memory once the stream has passed the call
 *     (vd_synchronize).  Calls that write to host memory synchronise the
 *     context's stream before returning.
 *   - Work is queued on the context's stream (vd_set_stream) and runs
 *     asynchronously.  A context is not thread-safe.
 *   - Every int-returning call returns VD_OK (0) or a negative VD_E* code and
 *     then leaves a message for vd_last_error() (per host thread).  A CUDA
 *     launch or copy error returns VD_ECUDA; the context should then be
 *     destroyed.
 */
#ifndef VD_H_
#define VD_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VD_OK 0
#define VD_EINVAL (-1)   /* bad argument: null handle, size or coordinate out of range */
#define VD_ENOMEM (-2)   /* device allocation failed */
#define VD_ECUDA (-3)    /* a CUDA runtime call or kernel launch failed */
#define VD_ETIMEOUT (-4) /* a bounded wait in a persistent kernel expired */
#define VD_EBUSY (-5)    /* resource exhausted (serving: no slot or budget) */
#define VD_ENOTFOUND (-6) /* unknown id (serving) */

#define VD_METRIC_EUCLID 0
#define VD_METRIC_MANHATTAN 1
#define VD_NB_MOORE 0
#define VD_NB_VON_NEUMANN 1

#define VD_MAX_SIDE 32768
#define VD_MAX_PASSES 64

/* Message of the last failing call on this host thread ("" if none). */
const char* vd_last_error(void);

/* ABI version of this header (increments on any incompatible change). */
int vd_abi_version(void);

/* ------------------------------------------------------------------------ */
/* Schedules (host arithmetic, no GPU needed)                               */
/* ------------------------------------------------------------------------ */

/*
 * JFA step lengths, Eq. 2 (Section III): k_1 = 2^(ceil(log2 N) - 1) with
 * N = max(w, h), then k_1/2, ..., 1 (log2(k_1) + 1 passes; none when N = 1),
 * followed by `extra_passes` passes: 1 -> (1) [JFA+1], 2 -> (2, 1) [JFA+2].
 * Writes up to `cap` entries to ks (step lengths) and nbs (VD_NB_* per pass;
 * all Moore, Table I).  Returns the full pass count (may exceed cap), or
 * VD_EINVAL for bad sizes, extra_passes outside [0, 2] or null arrays with
 * cap > 0.
 */
int vd_jfa_schedule(int32_t w, int32_t h, int32_t extra_passes, int32_t* ks, int32_t* nbs,
                    int32_t cap);

/*
 * dJFA step lengths, Eq. 3-4 (Section V-A): delta_1 = 2^ceil(log2(max(
 * 2 L_avg, d_max))) with L_avg = sqrt(w h / s), decided in exact integers
 * (the least P = 2^e with P^2 s >= 4 w h and P >= d_max), capped at JFA's
 * k_1 (Algorithm 1's k_m).  Passes delta_1, ..., 1 (log2(delta_1) + 1), the
 * first `vn_waves` with the Von Neumann neighbourhood and the rest Moore
 * (Section V-B), then `extra_passes` as in vd_jfa_schedule (the optional
 * extra step after Eq. 4).  Same output and errors as vd_jfa_schedule;
 * vn_waves must be >= 0.
 */
int vd_djfa_schedule(int32_t w, int32_t h, int64_t n_seeds, int32_t d_max, int32_t vn_waves,
                     int32_t extra_passes, int32_t* ks, int32_t* nbs, int32_t cap);

/* ------------------------------------------------------------------------ */
/* One simulation                                                            */
/* ------------------------------------------------------------------------ */

typedef struct vd_ctx vd_ctx;

/*
 * Creates a simulation on the current CUDA device: the state that Algorithm 1
 * threads through its steps, Data = (VD, S, A) -- the label map VD of the
 * problem statement in Section IV (the discrete diagram of a w x h grid, one
 * seed index per pixel), the seed set S and the step count -- as a w x h label
 * map (two
 * device buffers for the Jacobi passes, rows padded to 128 bytes, the
 * padding held at -1), n_seeds seeds (all at (0, 0) until vd_set_seeds) and
 * small scratch buffers.  Labels start at -1.  The stream is the legacy
 * default stream until vd_set_stream.  Returns NULL on bad sizes (w, h
 * outside [1, VD_MAX_SIDE], n_seeds < 1) or allocation failure
 * (vd_last_error() says which).
 */
vd_ctx* vd_create(int32_t grid_w, int32_t grid_h, int32_t n_seeds);

/* Ends a simulation (the Data = (VD, S, A) of Algorithm 1 that vd_create
 * made): frees every device buffer of the context after its stream is idle.
 * NULL is accepted (VD_OK). */
int vd_destroy(vd_ctx* ctx);

/* Queues all later work of the context on `cuda_stream` (a cudaStream_t;
 * NULL = legacy default stream).  The caller keeps the stream alive.  The
 * paper runs every step of Algorithm 1 on one GPU (Section VI); the stream is
 * where this library orders those steps.  VD_EINVAL on a null context. */
int vd_set_stream(vd_ctx* ctx, void* cuda_stream);

/* Blocks until all queued work of the context has finished. */
int vd_synchronize(vd_ctx* ctx);

/* Grid and seed sizes of a context (any output pointer may be NULL). */
int vd_get_shape(const vd_ctx* ctx, int32_t* w, int32_t* h, int32_t* n_seeds,
                 int32_t* row_pitch);

/*
 * Replaces the seed positions with n_seeds (x, y) pairs (Section II, the set
 * S).  VD_EINVAL if any coordinate lies outside the grid (checked on the
 * host for host input, on the device for device input, where the check
 * costs a synchronisation).
 */
int vd_set_seeds(vd_ctx* ctx, const int32_t* xy, int on_device);

/* Copies the current seed positions out (n_seeds pairs). */
int vd_get_seeds(vd_ctx* ctx, int32_t* xy, int on_device);

/*
 * SimulateParticles of Algorithm 1 under the uniform random model of
 * Section V-A: every seed k moves to clamp(p_k + delta_k) with the clamp
 * keeping it on the grid.  If dxy is non-NULL it holds n_seeds integer
 * displacement pairs (host or device per dxy_on_device, a device pointer
 * 8-byte aligned; max_disp, rng_seed, stream_id and step are then ignored).  If dxy is NULL, each displacement
 * component is drawn on the device as u - max_disp, u uniform in
 * [0, 2 max_disp] from SplitMix64 (Steele, Lea, Flood 2014): key =
 * splitmix64(rng_seed, stream_id), draw = splitmix64(key, step * 2^33 + 2k +
 * axis), u = ((draw >> 32) * (2 max_disp + 1)) >> 32, where splitmix64(s, n)
 * is the n-th output of the generator started at state s.  VD_EINVAL if
 * max_disp < 0 or > VD_MAX_SIDE (RNG mode) or step < 0.
 */
int vd_move_seeds(vd_ctx* ctx, const int32_t* dxy, int dxy_on_device, int32_t max_disp,
                  uint64_t rng_seed, uint64_t stream_id, int64_t step);

/*
 * Seed removal and insertion between frames.  The paper leaves both to future
 * work (Section VII); the rule here is this library's own:
 *   - the seeds whose indices are listed in remove_ids (n_remove distinct
 *     indices in [0, n)) leave; the survivors keep their order and are
 *     renumbered 0 .. n - n_remove - 1;
 *   - the n_add seeds of add_xy (x, y pairs on the grid) follow them;
 *   - the current label map is relabelled: a surviving seed's pixels take its
 *     new index, a removed seed's pixels become empty (-1);
 *   - after any removal, the next vd_djfa_step runs the full JFA schedule
 *     (Eq. 2, plus its `extra` passes) on the relabelled map instead of the
 *     dJFA schedule, so the emptied cells fill from every side whatever their
 *     size; after insertions only, the dJFA schedule runs (a new seed is
 *     stamped and claims its cell like a moved one).  vd_jfa clears this.
 * The seed count may grow past the one given to vd_create (the seed buffers
 * are reallocated, synchronously); at least one seed must remain.  Both
 * arrays are host (on_device = 0) or device pointers; they are copied.
 * Returns VD_EINVAL, changing nothing, for an index out of range or repeated,
 * a new seed off the grid, or no seed left.  Host inputs are validated on the
 * host and the update is queued on the stream; device inputs are validated on
 * the device, which synchronises the stream once.  Growing past the
 * allocation synchronises too.
 */
int vd_update_seeds(vd_ctx* ctx, const int32_t* remove_ids, int32_t n_remove, const int32_t* add_xy,
                    int32_t n_add, int on_device);

/*
 * A full JFA frame (Section III): empties the map (-1), stamps the seeds
 * (each seed pixel gets the lowest index standing on it) and runs the passes
 * of vd_jfa_schedule with the Moore neighbourhood of Table I.  Each pass is
 * a gather: pixel q keeps, among itself and its in-grid neighbours at
 * offset k that hold a label, the seed nearest to q (lowest index on ties),
 * reading one buffer and writing the other.  VD_EINVAL for a bad metric or
 * extra_passes outside [0, 2].
 */
int vd_jfa(vd_ctx* ctx, int32_t extra_passes, int32_t metric);

/*
 * One dJFA frame (Section V, Algorithm 1 after SimulateParticles): stamps
 * the current seeds onto the previous frame's map without clearing it, then
 * runs the passes of vd_djfa_schedule(w, h, n_seeds, d_max, vn_waves,
 * extra_passes).  d_max is the per-step move bound of Section V-A (the
 * Chebyshev bound of the moves, e.g. max_disp).  VD_EINVAL for d_max < 0,
 * vn_waves < 0, bad metric or extra_passes outside [0, 2].
 */
int vd_djfa_step(vd_ctx* ctx, int32_t d_max, int32_t vn_waves, int32_t extra_passes,
                 int32_t metric);

/*
 * One whole timestep (Algorithm 1's loop body): the move of vd_move_seeds
 * (same arguments, same result) followed by the frame of vd_djfa_step (same
 * arguments; the repair schedule after a removal).  With VD_OPT_USE_GRAPHS
 * the whole step replays as one graph whose move arguments are replaced every
 * call.  Results equal vd_move_seeds + vd_djfa_step bit for bit.
 */
int vd_step(vd_ctx* ctx, const int32_t* dxy, int dxy_on_device, int32_t max_disp, uint64_t rng_seed,
            uint64_t stream_id, int64_t step, int32_t d_max, int32_t vn_waves, int32_t extra, int32_t metric);

/* The stamp alone (part of vd_jfa / vd_djfa_step): every seed pixel of the
 * current map gets the lowest index among the seeds standing on it. */
int vd_stamp(vd_ctx* ctx);

/* One jump pass with step k >= 1 and neighbourhood nb (Table I for Moore,
 * Section V-B for Von Neumann), as inside vd_jfa; exposed for tests and
 * diagnostics. */
int vd_pass(vd_ctx* ctx, int32_t k, int32_t nb, int32_t metric);

/*
 * One jump pass (as vd_pass) that computes only rows [y0, y1) of the next
 * map, reading rows y0 - k .. y1 - 1 + k of the current one; the other rows
 * of the next map keep whatever they held.  This is the per-band step of a
 * map split into row bands across GPUs (each GPU owns one band and, before
 * every pass, receives from the others the rows y0 - k .. y0 - 1 and
 * y1 .. y1 - 1 + k its band reads -- for JFA's first steps k exceeds the
 * band height, so they come from bands further away).  The pass reads its
 * neighbours k rows away (Table I, Section V-B), so a band's halo is k rows
 * deep; Eq. 4 bounds dJFA's largest step, and with it the halo.  djfa_frame
 * = 1 picks the key forms of a dJFA frame's passes, 0 those of a JFA frame
 * (results never depend on it).  VD_EINVAL for a bad step, neighbourhood,
 * metric or row range (0 <= y0 < y1 <= h).
 */
int vd_pass_rows(vd_ctx* ctx, int32_t k, int32_t nb, int32_t metric, int32_t y0, int32_t y1, int32_t djfa_frame);

/* Empties the current map (label -1 everywhere): the first step of a JFA
 * frame (Section III), for frames assembled from vd_stamp and vd_pass_rows. */
int vd_clear_labels(vd_ctx* ctx);

/* Overwrites the label map with a dense w x h map.  Every label must lie in
 * [-1, n_seeds): VD_EINVAL otherwise (checked on the host for host input, by a
 * kernel plus a synchronisation for device input) and the map is unchanged. */
int vd_set_labels(vd_ctx* ctx, const int32_t* labels, int on_device);

/* Copies the label map out as a dense w x h map: VD, the discrete Voronoi
 * diagram that Algorithm 1 returns each step (Section IV states the problem as
 * producing it every frame).  Host output synchronises the stream first. */
int vd_get_labels(vd_ctx* ctx, int32_t* labels, int on_device);

/*
 * Asynchronous read-back of the current label map into a dense w x h HOST
 * buffer, for pipelines that overlap the copy with the next frames: the map
 * is snapshotted on the context's stream (so later frames may rewrite it) and
 * copied out on a copy stream of the context.  Returns at once; the copy is
 * complete when vd_wait_labels returns.  Two copies may be outstanding; a
 * third call first waits for the oldest.  `labels` should be page-locked for
 * the copy to overlap, and must stay valid until the wait.  Allocates two
 * snapshot maps on first use.
 */
int vd_get_labels_async(vd_ctx* ctx, int32_t* labels);
/*
 * As vd_get_labels_async, into a dense w x h map of 16-bit labels (half the
 * bytes to copy): each label as it is, the empty label -1 as 0xFFFF.  Needs
 * at most 65535 seeds (VD_EINVAL otherwise).  The map is narrowed on the
 * context's stream into one of the same two snapshot slots, so the two calls
 * share the limit of two outstanding copies.
 */
int vd_get_labels16_async(vd_ctx* ctx, uint16_t* labels);
/*
 * As vd_get_labels_async, into a dense w x h map of 24-bit labels, three
 * little-endian bytes each (3/4 of the bytes to copy; labels the host can
 * widen or use as they are): each label as it is, the empty label -1 as
 * 0xFFFFFF.  `labels` holds 3 * w * h bytes.  Needs at most 16777215 seeds
 * (VD_EINVAL otherwise).  Packed on the context's stream into one of the
 * same two snapshot slots as the other asynchronous read-backs.
 */
int vd_get_labels24_async(vd_ctx* ctx, uint8_t* labels);
/*
 * As vd_get_labels_async, into a dense bit stream of `bits`-bit labels
 * (bits in [1, 32]; the fewest bytes to copy, for pipelines bound by the
 * host link): label j = y * w + x occupies bits [j * bits, (j + 1) * bits)
 * of the stream, least significant bit first within little-endian bytes,
 * the empty label -1 as 2^bits - 1.  `labels` holds ceil(w * h * bits / 8)
 * bytes.  Needs at most 2^bits - 1 seeds (VD_EINVAL otherwise), so that no
 * label takes the empty code; the fewest bits for n seeds are the bit length
 * of n.  Packed on the context's stream into one of the same two snapshot
 * slots as the other asynchronous read-backs.
 */
int vd_get_labels_packed_async(vd_ctx* ctx, uint8_t* labels, int32_t bits);
/* Waits until every vd_get_labels_async / vd_get_labels16_async /
   vd_get_labels24_async / vd_get_labels_packed_async copy of the context
   has landed. */
int vd_wait_labels(vd_ctx* ctx);

/*
 * Borrowed device pointer to the current label map (row pitch in elements
 * via vd_get_shape); valid until the next call on the context.
 */
int vd_labels_device_ptr(vd_ctx* ctx, const int32_t** labels);

/*
 * Similarity counts of Section VI-A for the current map against optional
 * dense references (host or device per on_device):
 *   n_match = #pixels whose label equals ref_labels (the paper's similarity
 *             is 100 n_match / (w h) against a same-frame JFA);
 *   n_exact = #pixels whose label's seed is at distance exact_dist from the
 *             pixel, exact_dist being the exact minimum distance of Eq. 1 in
 *             `metric` (the distance-correct count).
 * A NULL reference gives a count of 0.  Synchronises (results on the host).
 */
int vd_similarity(vd_ctx* ctx, const int32_t* exact_dist, const int32_t* ref_labels,
                  int on_device, int32_t metric, uint64_t* n_exact, uint64_t* n_match);

/* n_match of the current maps of two contexts of the same grid size. */
int vd_similarity_ctx(vd_ctx* ctx, vd_ctx* ref, uint64_t* n_match);

/*
 * The exact diagram of Eq. 1 on the device: for every pixel the lowest seed
 * index at the minimum distance (labels) and that distance (dist), each
 * written as a dense w x h map when non-NULL (host or device per on_device).
 * Exact by construction (a uniform bucket grid searched ring by ring until
 * no unvisited bucket can hold a seed at distance <= the best).  Does not
 * touch the context's label map.
 */
int vd_exact(vd_ctx* ctx, int32_t* labels, int32_t* dist, int on_device, int32_t metric);

/*
 * Exact diagram for callers that cannot allocate device memory.  The paper has
 * no counterpart to this call; it exists for code that must not call
 * cudaMalloc: code running under another framework's memory manager (which
 * owns the device memory and budgets every byte of it), latency-bound loops
 * that cannot afford the synchronisation an allocation may bring, and plugin
 * hosts that forbid allocation on their threads.  vd_exact needs a context,
 * and a context allocates; this entry point takes everything as caller
 * buffers and uses a fixed scratch array compiled into the library instead.
 *
 * Computes the same maps as vd_exact: for every pixel of a w x h grid the
 * lowest seed index at the minimum distance (labels) and that distance
 * (dist), dense row-major int32, either may be NULL but not both.  seeds_xy,
 * labels and dist are DEVICE pointers of the current device (seeds_xy 8-byte
 * aligned, n_seeds (x, y) pairs); the caller owns them.  Work runs on
 * cuda_stream (NULL = legacy default stream); the call first synchronises
 * that stream once to check the seeds, then queues the rest and returns.
 *
 * Scratch: a file-scope device array of VD_NOALLOC_SCRATCH_INTS int32 (4 MiB)
 * that every GPU loading the library holds until the process exits.  The
 * bucket grid needs 64 + 2 * buckets + 1 + n_seeds ints, and the bucket side
 * is chosen so that there are at most two buckets per seed, so the need is at
 * most 66 + 5 * n_seeds ints: up to 200000 seeds always fit, on any grid.
 * Larger requests fail with VD_EINVAL and a message naming the need, as do
 * bad sizes, a bad metric and seeds outside the grid.  No cudaMalloc,
 * cudaFree or allocating library routine is called.  Every call synchronises
 * the stream for the seed check, so the call cannot be captured into a CUDA
 * graph.  The array's device address is resolved on every call (with the
 * seeds' device current), so it stays valid across a device reset.  All calls
 * share the one array, which keeps the previous call's contents (the parts
 * that must start at zero are cleared on every call): calls that overlap on
 * the GPU, on any stream, race.
 */
#define VD_NOALLOC_SCRATCH_INTS (1 << 20)
int vd_exact_noalloc(const int32_t* seeds_xy, int32_t n_seeds, int32_t grid_w, int32_t grid_h,
                     int32_t metric, int32_t* labels, int32_t* dist, void* cuda_stream);

/* ------------------------------------------------------------------------ */
/* Many independent simulations (batched timestep)                          */
/* ------------------------------------------------------------------------ */

/*
 * A batch steps many independent simulations (each its own grid and seeds)
 * together.  Every simulation computes exactly what a context would compute
 * for it alone (vd_jfa, vd_move_seeds with stream_id = its index,
 * vd_djfa_step): the same per-pixel code, the same exact-integer results.
 * The paper runs one simulation at a time (Section VI); batching is this
 * library's way of filling a GPU with many small grids.
 */
typedef struct vd_batch vd_batch;

/*
 * Creates a batch of n_sims simulations with grid sizes w[i] x h[i] and
 * n_seeds[i] seeds (host arrays; sizes as for vd_create).  All label maps
 * start empty (-1), all seeds at (0, 0).  Seed arrays of the batch are
 * concatenated in simulation order ("sim-major"): simulation i's seeds start
 * at the offset vd_batch_get_shape reports.  NULL on bad sizes or OOM.
 */
vd_batch* vd_batch_create(int32_t n_sims, const int32_t* w, const int32_t* h, const int32_t* n_seeds);
int vd_batch_destroy(vd_batch* batch);
int vd_batch_set_stream(vd_batch* batch, void* cuda_stream);

/* Waits for the batch's stream.  Returns VD_ETIMEOUT (once, then clears it)
 * if a persistent step's bounded barrier wait ran out since the last check;
 * the maps of that step are then undefined (re-run vd_batch_jfa). */
int vd_batch_synchronize(vd_batch* batch);

/* Grid size, seed count and seed offset of simulation `sim`. */
int vd_batch_get_shape(const vd_batch* batch, int32_t sim, int32_t* w, int32_t* h, int32_t* n_seeds,
                       int32_t* seed_offset);

/* Replaces all seeds (sim-major (x, y) pairs, total = sum of n_seeds);
 * VD_EINVAL if any lies outside its simulation's grid (nothing changes). */
int vd_batch_set_seeds(vd_batch* batch, const int32_t* xy, int on_device);
int vd_batch_get_seeds(vd_batch* batch, int32_t sim, int32_t* xy, int on_device);
/* Dense w x h label map of one simulation (synchronises the batch). */
int vd_batch_get_labels(vd_batch* batch, int32_t sim, int32_t* labels, int on_device);

/* Sets the dJFA schedule of every simulation (Eq. 3-4 with its own w, h,
 * n_seeds; parameters as vd_djfa_step).  Needed before vd_batch_step. */
int vd_batch_configure(vd_batch* batch, int32_t d_max, int32_t vn_waves, int32_t extra_passes,
                       int32_t metric);

/* A full JFA frame (Section III) for every simulation, e.g. frame 0. */
int vd_batch_jfa(vd_batch* batch, int32_t metric);

/*
 * One dJFA timestep of every simulation: move (given sim-major displacements
 * dxy, or SplitMix64 draws in [-max_disp, max_disp] with stream_id = the
 * simulation's index and step = the number of moves it has made so far, as
 * in vd_move_seeds), stamp onto the previous map, and the configured passes.
 * In the default mode every phase and pass round is one launch over all
 * simulations' tiles, the whole step replayed as a CUDA graph once its plan
 * repeats; in VD_BMODE_PERSISTENT it is one cooperative launch with a bounded
 * grid barrier between phases (see vd_batch_synchronize).
 */
int vd_batch_step(vd_batch* batch, const int32_t* dxy, int dxy_on_device, int32_t max_disp,
                  uint64_t rng_seed);

/* The same timestep for a subset of simulations only (RNG moves; each listed
 * at most once), e.g. the requests a server admitted together. */
int vd_batch_step_subset(vd_batch* batch, const int32_t* sims, int32_t n, int32_t max_disp,
                         uint64_t rng_seed);

#define VD_BOPT_MODE 1               /* 0 = launch per phase/round (default), 1 = persistent */
#define VD_BOPT_ROWS_PER_THREAD 2    /* rows each thread sweeps per tile: 1 (default), 2, 4, 8, 16 */
#define VD_BOPT_BLOCKS_PER_SM 3      /* persistent mode: 0 = occupancy maximum (default), else cap */
#define VD_BOPT_USE_GRAPHS 4         /* 1 (default) = replay repeating full steps as a graph */
#define VD_BOPT_BARRIER_TIMEOUT_US 5 /* persistent mode: bounded barrier wait (default 2 s) */
#define VD_BOPT_TEST_SKIP_ARRIVE 6   /* test only: block 0 skips its first barrier arrival so the
                                        other blocks' wait must run out (default 0) */
#define VD_BOPT_CLAMPED_KEYS 7       /* as VD_OPT_CLAMPED_KEYS (-1 auto, 0 never, 1 always when usable);
                                        applied at the next vd_batch_configure / vd_batch_jfa */
#define VD_BOPT_PERSISTENT_BYTE_KEYS 8 /* persistent mode: 1 (default) = the byte-offset key on the passes
                                        whose simulations the auto rules give it, as the per-round
                                        launches do; 0 = the clamped key there.  Results never depend
                                        on it */
#define VD_BOPT_PERSISTENT_MIN_BLOCKS 9 /* persistent mode: register budget of the kernel, 4 (default, 64
                                        registers a thread) or 5 (48) resident 256-thread blocks per SM */
#define VD_BOPT_PACKED_MAP 10        /* launch per round: -1 (default) = a simulation's dJFA frame runs its
                                        last passes (at least two, k = 1, 2 or a multiple of 4 up to
                                        128) on position-tagged words, as VD_OPT_PACKED_MAP does for
                                        one simulation, where it has up to 32767 seeds and mean cells
                                        of radius at most 40 pixels; 0 = never.  Takes effect at the
                                        next vd_batch_configure.  The persistent mode runs every pass
                                        on labels.  Results never depend on it */
int vd_batch_set_option(vd_batch* batch, int32_t option, int64_t value);
int vd_batch_get_option(const vd_batch* batch, int32_t option, int64_t* value);

/*
 * Autotuner: times `steps` dJFA steps (after one warm-up step) for each
 * candidate launch shape, restoring the batch's
 * complete state (maps, seeds, step counters) before each candidate and at
 * the end, so tuning leaves the simulation unchanged.  Keeps the fastest
 * candidate; writes its index to *best and each candidate's ms per step to
 * ms_per_step[0 .. cap).  Returns the number of candidates.  The candidates,
 * in order (mode, rows per thread, blocks per SM): per-round launches with 1,
 * 2 or 4 rows per thread (tiles of 256 x 4, 8 or 16 pixels) [0-2]; the
 * persistent launch with 1, 2 or 4 rows per thread at the occupancy maximum
 * [3-5]; the persistent launch with 1 or 2 rows per thread capped at 3 blocks
 * per SM [6-7] and at 2 [8-9]; the persistent launch with 1 or 2 rows per
 * thread on the clamped key only (VD_BOPT_PERSISTENT_BYTE_KEYS = 0) [10-11];
 * the persistent launch with 1, 2 or 4 rows per thread compiled for 5
 * blocks per SM (VD_BOPT_PERSISTENT_MIN_BLOCKS = 5) [12-14]; per-round
 * launches with 8 or 16 rows per thread (tiles of 256 x 32 or 64) [15-16].
 */
int vd_batch_autotune(vd_batch* batch, int32_t steps, int32_t max_disp, uint64_t rng_seed,
                      int32_t* best, double* ms_per_step, int32_t cap);

/* Total pixels, pixel-passes of one configured dJFA step, total seeds. */
int vd_batch_work(const vd_batch* batch, int64_t* pixels, int64_t* pixel_passes_per_step,
                  int64_t* seeds);
int64_t vd_batch_launch_count(const vd_batch* batch);

/* ------------------------------------------------------------------------ */
/* Serving: resident simulations, step requests, continuous batching        */
/* ------------------------------------------------------------------------ */

/*
 * A server keeps up to max_sims simulations resident on the device (maps,
 * seeds and seed table in one allocation each), admitting a simulation only
 * while the total stays within hbm_budget_bytes.  Clients submit dJFA step
 * requests; each request moves the simulation's seeds by SplitMix64 draws in
 * [-max_disp, max_disp] (stream_id = the simulation's id, step = the number of
 * steps it has taken, as in vd_move_seeds) and runs one dJFA frame with the
 * server's d_max, vn_waves and metric (as vd_djfa_step).  Requests are served
 * in arrival order with continuous batching: two launch lanes (own stream,
 * plan and completion event each) alternate, and a free lane takes every
 * queued request whose simulation has no step in flight, so newly arrived
 * requests join the next launch while the previous one still runs.  A
 * simulation's result is the same alone or in any mix.  The paper has no
 * serving layer; this is the library's own.  A server is not thread-safe.
 */
typedef struct vd_server vd_server;

vd_server* vd_server_create(int32_t max_sims, int64_t hbm_budget_bytes, int32_t d_max, int32_t vn_waves,
                            int32_t metric, int32_t max_disp, uint64_t rng_seed);
int vd_server_destroy(vd_server* server);

/*
 * Admits a simulation (host seeds, n (x, y) pairs), runs its JFA frame 0 and
 * returns its id (>= 0).  VD_EBUSY if it would exceed the HBM budget or all
 * slots are live (the message gives the shortfall), VD_EINVAL for bad sizes
 * or seeds, VD_ENOMEM if the device allocation fails.
 */
int32_t vd_server_add_sim(vd_server* server, int32_t w, int32_t h, int32_t n_seeds, const int32_t* xy);
/* Frees a simulation's memory and budget (VD_EBUSY while it has work). */
int vd_server_remove_sim(vd_server* server, int32_t sim);

/* Queues one step request; t_arrive (seconds on the server clock,
 * vd_server_now) is the time latency is measured from, or < 0 for now.
 * Returns the request's ticket (>= 0). */
int64_t vd_server_submit(vd_server* server, int32_t sim, double t_arrive);
/* Reaps finished launches and admits queued requests into free lanes;
 * returns the number of requests completed by this call.  Never blocks. */
int vd_server_progress(vd_server* server);
/* Runs progress until nothing is queued or in flight. */
int vd_server_drain(vd_server* server);
/* Moves up to cap completion records out (ticket, latency in seconds,
 * simulation; any array may be NULL); returns how many. */
int32_t vd_server_completions(vd_server* server, int64_t* tickets, double* latency_s, int32_t* sims,
                              int32_t cap);
/* Seconds since the server was created (its clock). */
double vd_server_now(const vd_server* server);
/*
 * Replays a timed trace natively: request i for simulation sims[i] arrives
 * arrival_s[i] seconds after the call starts (non-decreasing); the call
 * submits each at its time, keeps the lanes busy, and returns when all are
 * done with each request's latency (completion - scheduled arrival).
 */
int vd_server_run_trace(vd_server* server, const double* arrival_s, const int32_t* sims, int64_t n,
                        double* latency_s);
/* Dense label map of a simulation (waits for its in-flight step). */
int vd_server_get_labels(vd_server* server, int32_t sim, int32_t* labels, int on_device);
int vd_server_stats(const vd_server* server, int64_t* used_bytes, int64_t* budget_bytes, int32_t* live_sims,
                    int64_t* pending, int64_t* steps_done, int64_t* launches);
/* Caps the requests one launch may take (default unbounded). */
int vd_server_set_max_batch(vd_server* server, int32_t max_batch);

/* Tuning and execution options (vd_set_option); values are validated. */
#define VD_OPT_FUSE_MAX_K 1      /* largest step fused into shared-memory groups (0 = no fusion, the
                                    default; 1..16) */
#define VD_OPT_BAND_ORDER_MIN_K 2 /* step from which large-k passes visit rows in k-strided bands (0 = never) */
#define VD_OPT_USE_GRAPHS 3      /* 1 = replay each frame's launches as a cached CUDA graph */
#define VD_OPT_FUSE_TILE_X 4     /* fused-group tile width in pixels (multiple of 4, 16..256) */
#define VD_OPT_FUSE_TILE_Y 5     /* fused-group tile height in pixels (1..128) */
#define VD_OPT_PROFILE 6         /* 1 = bracket every kernel launch with CUDA events (frames then run
                                    eagerly, never from a graph); read with vd_profile_read */
#define VD_OPT_CLAMPED_KEYS 7    /* passes with one 32-bit key per candidate, all exact:
                                    Euclidean min(d^2, cap) * 2^lb + label and, beyond 32768 seeds,
                                    Manhattan min(d, cap) * 2^lb + label (cap = 2^(32 - lb) - 1; quads
                                    that reach the cap are recomputed with the 64-bit key; usable
                                    with >= 9 seeds); up to 32768 seeds Manhattan d * 2^lb + label
                                    (no cap).  -1 = auto (default: clamped keys for dJFA passes, the
                                    uncapped Manhattan key for every pass), 0 = never, 1 = always
                                    when usable */
#define VD_OPT_PDL 8             /* 1 (default) = a frame's stamp and pass kernels are chained with
                                    programmatic dependent launch: each may be scheduled while its
                                    predecessor drains and waits for it on the device before touching
                                    memory; 0 = plain stream order.  Results never depend on it */
#define VD_OPT_DEDUP_GATHERS 9   /* a label equal to its left neighbour in a 4-label vector reuses that
                                    neighbour's table gather: -1 = auto (default: dJFA passes on maps
                                    of at most 256 pixels per seed), 0 = never, 1 = always.  Results
                                    never depend on it */
#define VD_OPT_BYTE_KEYS 10      /* Euclidean passes with the byte-offset key: one dp4a of the packed
                                    seed-minus-pixel offset gives d^2, exact for dx, dy in [-h, h)
                                    (h = 128 below 65536 seeds; from 65536 seeds on the label field
                                    widens and h narrows: 64 .. 32 below 2^20 seeds, 16 .. 8 at up
                                    to 2^22); each pixel's winner is checked against that window and
                                    a failing quad is recomputed with the clamped key, so results
                                    are exact.  -1 = auto (default: dJFA passes with steps up to
                                    min(128, 2h) on maps of at least 2^21 pixels whose mean cell
                                    radius is at most 40 h / 128 pixels, with h >= 32), 0 = never,
                                    1 = always when usable (>= 9 seeds) */
#define VD_OPT_BLOCKED_PASS 11   /* byte-key passes with k a multiple of 4 run register-blocked: one
                                    thread owns the four quads at (x, y), (x + k, y), (x, y + k),
                                    (x + k, y + k), whose neighbour vectors overlap, and loads and
                                    gathers each of the 16 (Moore) or 12 (Von Neumann) vectors once.
                                    -1 = auto (default: never; it measured slower than the plain pass
                                    on the GB300, where the pass is bound on integer issue and the
                                    blocked form runs at half the occupancy), 0 = never, 1 = whenever
                                    it applies.  Results never depend on it */
#define VD_OPT_KEY_PACK 12       /* how the blocked byte-key pass packs (d, label): 0 = multiply-add
                                    (default), 1 = byte permute (below 2^16 seeds), 2 = constant shift
                                    (2^16 seeds and more).  Results never depend on it */
#define VD_OPT_BLOCKED_MIN_BLOCKS 13 /* register budget of the blocked pass: 8 (default, 64 registers a
                                    thread) or 6 (80) resident 128-thread blocks per SM */
#define VD_OPT_SPARSE_PASS 14    /* passes with k % 4 == 0, k = 1 or k = 2 first test each quad: when
                                    every in-grid candidate of each of its pixels carries the pixel's
                                    own label the quad is copied through; the other quads of the block
                                    are gathered in shared memory and scored one per thread.  -1 = auto
                                    (default: steps of at most 1/32 of the mean cell side
                                    sqrt(w h / n), where nearly every quad is unchanged), 0 = never,
                                    1 = whenever it applies.  Results never depend on it */
#define VD_OPT_JFA_POSITION_MAP 15 /* the passes of a JFA frame with k % 4 == 0 read and write a map of
                                    (label, packed position) pairs, so that a candidate's position comes
                                    with its label and nothing is gathered (JFA's middle passes, where
                                    neighbouring pixels name unrelated distant seeds, are otherwise
                                    bound by scattered table reads); 16 bytes a pixel per pass instead
                                    of 8, two such maps allocated on first use.  -1 = auto (default:
                                    maps of at least 2^20 pixels), 0 = never, 1 = always.  Results
                                    never depend on it */
#define VD_OPT_PASS_TILE 16      /* block tile of the jump pass: 128 threads as 64 quads (256 pixels) x 2
                                    rows (default), 32 x 4 or 128 x 1.  Results never depend on it */
#define VD_OPT_SMEM_TILE_MAX_K 17 /* byte-key passes with k = 1, 2 or a multiple of 4 up to this value
                                    (0 = never (default), 1, 2, 4, 8, 16) run over a shared-memory tile:
                                    each block of 256 x 16 pixels stages its tile and a k-pixel halo
                                    as (label, seed position) pairs, one table read per staged pixel,
                                    then reads every candidate from shared memory.  It measured
                                    slower than the plain pass with large seed tables (the tile
                                    takes most of L1) and about even with small ones, so it is
                                    opt-in.  Results never depend on it */
#define VD_OPT_SMEM_TILE_ROWS 18 /* rows of that tile: 16 (default, 1024-thread blocks) or 8 (512) */
#define VD_OPT_PACKED_MAP 19     /* dJFA frames whose last passes (at least two, each with k = 1, 2 or
                                    a multiple of 4) take the byte-offset key (up to 2^18 seeds) or
                                    the clamped key (2^18 + 1 to 2^22) run them on a
                                    position-tagged map: each 32-bit word holds the label and the
                                    low 8, 7, 6 or 4 bits of its seed's x and y (up to 32767 seeds,
                                    32768 to 2^17 - 1, 2^17 to 2^18, to 2^22), so that a candidate
                                    is scored with no table gather; the first of those passes reads
                                    the plain map and the last writes it again.  -1 = auto
                                    (default: the byte-offset key's mean-radius and step bounds
                                    with the layout's window 2^(M-1); with 4 bits also k times the
                                    frame's first step at most 64), 0 = never, 1 = whenever usable.
                                    Results never depend on it */
int vd_set_option(vd_ctx* ctx, int32_t option, int64_t value);

/*
 * Autotuner of the jump passes' launch shape for this context's dJFA frames
 * (the paper has no counterpart; the choices never change a result).  From a
 * device snapshot of the state (map, seeds, tables), each candidate setting
 * runs `steps` timed dJFA steps (vd_step with SplitMix64 moves in
 * [-max_disp, max_disp], stream 0, steps 0 .. steps - 1; d_max, vn_waves and
 * metric as for vd_djfa_step) after one untimed step; the snapshot is
 * restored before every candidate and at the end, so the state is left as it
 * was.  The search goes through one dimension at a time, the others held at
 * the best so far: the position-tagged passes (VD_OPT_PACKED_MAP -1, 0),
 * the pass block tile (VD_OPT_PASS_TILE 64, 32, 128),
 * gather de-duplication (VD_OPT_DEDUP_GATHERS -1, 0, 1), the sparse form
 * (VD_OPT_SPARSE_PASS -1, 0, 1), the register-blocked form
 * (VD_OPT_BLOCKED_PASS -1, 1) and, when on, its blocks per SM
 * (VD_OPT_BLOCKED_MIN_BLOCKS 8, 6), the shared-memory fusion depth of
 * small steps (VD_OPT_FUSE_MAX_K 0, 2, 4), the shared-memory tiled form
 * (VD_OPT_SMEM_TILE_MAX_K 0, 2, 8) and, when on, its rows
 * (VD_OPT_SMEM_TILE_ROWS 16, 8).  The fastest setting stays in force.
 * chosen (may be NULL) receives 9 values: the pass block tile, gather
 * de-duplication, the sparse form, the blocked form, its blocks per SM, the
 * fusion depth, the tiled form's largest step, its rows, then the
 * position-tagged passes; ms_per_step
 * (at least cap entries, may be NULL with cap = 0) the time of each candidate
 * measured, in order.  Allocates and frees one map-sized snapshot; synchronises
 * the stream.  Returns the number of candidates measured, or a VD_E* code
 * (the tuning is then left unchanged).
 */
int vd_autotune(vd_ctx* ctx, int32_t d_max, int32_t max_disp, int32_t vn_waves, int32_t metric, uint64_t rng_seed,
                int32_t steps, int32_t* chosen, double* ms_per_step, int32_t cap);
int vd_get_option(const vd_ctx* ctx, int32_t option, int64_t* value);

/* Kernel kinds reported by vd_profile_read. */
#define VD_KERNEL_PASS 0   /* one jump pass over the map (units: pixel-passes) */
#define VD_KERNEL_FUSED 1  /* a shared-memory group of small-step passes (units: pixel-passes) */
#define VD_KERNEL_STAMP 2  /* stamp halves (units: seeds) */
#define VD_KERNEL_MOVE 3   /* seed move (units: seeds) */
#define VD_KERNEL_FILL 4   /* map fill (units: pixels) */
#define VD_KERNEL_KINDS 5

/*
 * Profiling counters (VD_OPT_PROFILE = 1): synchronises the context's stream,
 * then adds up, per kernel kind, the GPU time between the events recorded
 * around each launch since the last vd_profile_reset.  Outputs (arrays of
 * VD_KERNEL_KINDS entries, any may be NULL): total milliseconds, launches and
 * work units.  VD_EINVAL if profiling is off.
 */
int vd_profile_read(vd_ctx* ctx, double* total_ms, int64_t* launches, int64_t* units);
int vd_profile_reset(vd_ctx* ctx);

/* Kernel launches issued by this context since creation (for accounting). */
int64_t vd_launch_count(const vd_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* VD_H_ */

/*
 * trk.h - C-ABI of the GB300 nested-geometry particle tracker.
 *
 * The library tracks neutral particles through nested constructive-solid-
 * geometry universes (arXiv 2406.13849): the find_cell /
 * distance_to_surface / move_within_cell / cross_surface loop of the
 * paper's Table 1, run inside run_histories (Alg. 2) with synthetic
 * physics.  Two trackers are built: a rect-array tracker chosen by static
 * dispatch (Alg. 5, 6, 9, 10) and a single CSG tracker whose universes,
 * arrays included, are CSG "pseudo-arrays" searched through a bounding
 * volume hierarchy over cell boxes (Sec. 4.3).
 *
 * Conventions for every entry point:
 *  - Plain pointers and sizes only.  "dev_" pointers are device memory on
 *    the current CUDA device, owned and allocated by the caller; the
 *    library allocates no device memory.  "host_" pointers are host memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Launches are asynchronous on it unless stated otherwise.
 *  - Calls return a trk_status and never throw.  On failure
 *    trk_last_error() returns a message (thread-local, valid until the next
 *    call from the same thread).
 *  - Failures found on the device (lost particles, segment caps, timeouts)
 *    are counted in the caller's counter array (TRK_K_*); a kernel-level
 *    failure also writes its status to counters[TRK_K_STATUS].
 *  - Sizes are validated on the host before any launch.
 */
#ifndef TRK_H
#define TRK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct trk_geom* trk_geom_t;   /* opaque, library-owned host object */

typedef enum {
    TRK_OK = 0,
    TRK_E_INVALID = -1,       /* bad argument (null pointer, size, option) */
    TRK_E_DESC = -2,          /* geometry description malformed or inconsistent */
    TRK_E_CUDA = -3,          /* a CUDA runtime call failed */
    TRK_E_NOMEM = -4,         /* caller buffer too small */
    TRK_E_LOST = -5,          /* particle lost (no cell where one must exist) */
    TRK_E_MAX_SEGMENTS = -6,  /* particle reached the segment cap */
    TRK_E_TIMEOUT = -7,       /* persistent kernel gave up after its iteration limit */
    TRK_E_UNSUPPORTED = -8,   /* option not supported for this geometry */
    TRK_E_SOURCE = -9         /* source rejection sampling exceeded its cap */
} trk_status;

/* Geometry descriptions may carry "accel": "bvh" (default) or "bih": the
 * acceleration structure of the CSG cell search, a BVH whose nodes hold both
 * children's boxes (64 B) or the bounding interval hierarchy of Sec. 4.3
 * (two bounding planes per node, 16 B).  Both return the same cells.
 *
 * Trackers.  RECT: the array tracker (static dispatch per universe type):
 * rect arrays by index (Alg. 5/6/9/10), hex arrays by a closed-form
 * element search checked against the element's pseudo-array cell (the paper
 * gives no hex array tracker; results are those of the pseudo-array scan),
 * CSG universes by search.  CSG: every array as its pseudo-array, searched
 * through a BVH of cell boxes (Sec. 4.3).  AUTO: CSG in event mode (its
 * kernel measured 1.25x RECT's on the 15 x 15 assembly core and within 6%
 * either way on a single pin lattice); in history mode and for the other
 * entry points RECT, or CSG for a geometry with hex arrays (measured as fast
 * or faster there).  DP: the paper's
 * dynamic-polymorphism method (Sec. 4.1), kept as a comparison: a rect array
 * tracker object and a CSG tracker object (hex arrays included) behind one
 * base class, every per-level find, distance and crossing a virtual call;
 * results equal RECT's.  run_histories (history mode, FP64, no mesh tally
 * or path cutoff; TRK_E_UNSUPPORTED otherwise) and trk_distance_to_surface
 * only; every other entry point rejects it with TRK_E_INVALID. */
enum { TRK_TRACKER_RECT = 0, TRK_TRACKER_CSG = 1, TRK_TRACKER_AUTO = 2, TRK_TRACKER_DP = 3 };
enum { TRK_MODE_HISTORY = 0, TRK_MODE_EVENT = 1 };
enum { TRK_FP64 = 0, TRK_FP32_LOCAL = 1 };

/* Counter slots (uint64 each, TRK_NCOUNTERS of them). */
enum {
    TRK_K_SEGMENTS = 0,     /* flights: surface crossings plus collision flights */
    TRK_K_CROSSINGS = 1,
    TRK_K_COLLISIONS = 2,
    TRK_K_ABSORBED = 3,
    TRK_K_ESCAPED = 4,
    TRK_K_REFLECTIONS = 5,
    TRK_K_LOST = 6,
    TRK_K_MAXSEG = 7,
    TRK_K_CUTOFF = 8,
    TRK_K_SOURCE = 9,
    TRK_K_CLOSE_CALLS = 10, /* FP32-local: decisions re-evaluated in FP64 */
    TRK_K_STATUS = 15,      /* first kernel-level trk_status (0 = none), two's complement */
    TRK_NCOUNTERS = 16
};

/* Per-particle terminal status written to records. */
enum { TRK_P_ALIVE = 0, TRK_P_ABSORBED = 1, TRK_P_ESCAPED = 2, TRK_P_CUTOFF = 3 };

typedef struct {
    int tracker;            /* TRK_TRACKER_* */
    int mode;               /* TRK_MODE_* */
    int precision;          /* TRK_FP64 or TRK_FP32_LOCAL */
    int block;              /* threads per block, 0 = default */
    int grid;               /* blocks, 0 = default (a multiple of the SM count) */
    int queue_depth;        /* event mode: particle slots per warp (32..512), 0 = default 256 */
    int sort_interval;      /* event mode: every sort_interval rounds each warp reorders its flight
                               queue by the class of the particles' leaf cells (no curved surface, one
                               cylinder from inside, from outside, other) so a flight batch runs one
                               code path; 0 = never (crossings are grouped by level every round) */
    int max_rounds;         /* event mode: round limit per warp, 0 = from max_segments; past it the
                               kernel stops and reports TRK_E_TIMEOUT in counters[TRK_K_STATUS] */
    uint64_t seed;          /* low 32 bits key the Philox stream with the geometry id */
    uint64_t first_id;      /* particle id of element 0 (ids key the random numbers; an id enters the
                               Philox counter as one 32-bit word, so ids are taken modulo 2^32 and
                               first_id + n <= 2^32 keeps every particle's stream distinct) */
    uint64_t max_segments;  /* per-particle segment cap (0 = 1e6) */
    double p_absorb;        /* absorption probability per collision */
    double max_path;        /* per-history path cutoff in cm (<= 0 or inf = none) */
    uint64_t* mesh_tally;   /* device uint64[mesh bins] (x fastest) or NULL: superimposed mesh
                               track-length tally, added to like the cell tally (the paper's active-
                               cycle flux tally); needs a mesh in the description, FP64, no cutoff */
} trk_run_opts;

/* Fills opts with the defaults: auto tracker, history mode, FP64, seed 1,
 * p_absorb 0.3, max_segments 1e6, no cutoff. */
void trk_default_opts(trk_run_opts* opts);

/* Message of the last failing call on this thread ("" if none). */
const char* trk_last_error(void);

/* Library build flavour: 1 if compiled with --fmad=false (every FP64
 * operation rounded once, in the order the method's formulas are written:
 * bit-exact against an FP64 evaluation of them), 0 for the fast build. */
int trk_exact_build(void);

/*
 * geometry_build - flatten a geometry description into device memory.
 * Sec. 1 (Table 1 and the universes of Fig. 3), Sec. 3.2 (coincident
 * lower-level surfaces removed), Sec. 4.3 (pseudo-array universes, cell
 * bounding boxes, SAH partitioning with three candidates per axis).
 *   json, len   description ("nested-csg-geometry-v1", see the package's
 *               inputs module), host memory, need not be NUL-terminated.
 *   dev_buf     device buffer of at least *dev_bytes bytes, 256-byte
 *               aligned; NULL to query the size only (then *dev_bytes is
 *               set, *out untouched).
 *   dev_bytes   in: capacity of dev_buf; out: bytes needed.
 *   stream      copies are enqueued on it; dev_buf must stay alive and
 *               unmodified until geometry_destroy.
 *   out         new handle (library-owned host object) on TRK_OK.
 * Errors: TRK_E_DESC (parse/validation, message says where), TRK_E_NOMEM
 * (dev_buf smaller than needed), TRK_E_INVALID, TRK_E_CUDA.
 */
trk_status geometry_build(const char* json, size_t len, void* dev_buf, size_t* dev_bytes,
                          void* stream, trk_geom_t* out);

/* Releases the host object (not the caller's device buffer).  NULL -> TRK_E_INVALID. */
trk_status geometry_destroy(trk_geom_t g);

/* Sizes of a built geometry: leaf cell instances (tally bins), materials,
 * maximum nesting depth, and whether the array tracker applies (always 1). */
trk_status geometry_info(trk_geom_t g, int64_t* n_instances, int32_t* n_materials,
                         int32_t* max_depth, int32_t* rect_ok);

/*
 * power_iteration - Alg. 1: `cycles` cycles of n histories, the first
 * `inactive` of them untallied, with a synthetic fission source.  The
 * description's optional "nu" (one value per material in [0, 7], 0 = none)
 * gives the fission yield: an absorption in material m with nu_m > 0 banks
 * floor(nu_m / k + xi) sites at the absorption point (at most 8; k the
 * previous cycle's estimate, 1 in the first cycle; xi from counter
 * (pid, e, 3, 0), e the absorbing collision).  Cycle 0 is born in the source
 * box, cycle c > 0 from cycle c-1's sites (kept in history order): particle
 * i of cycle c has id first_id + c*n + i and takes site floor(xi * B) (xi
 * from counter (pid, 0, 4, 0)), the direction and tau of source_init.
 *   dev_k      out: double[cycles], k_c = (double(sum of llrint(nu * 2^32)
 *              over the cycle's fissile absorptions) * 2^-32) / n
 *   dev_bank   out: int64[cycles], sites banked per cycle
 *   dev_tally, dev_counters: added to over the active cycles only
 *   dev_work   scratch of power_iteration_work_bytes (256-byte aligned):
 *              the particles, per-history sites, the bank (8n sites) and,
 *              in event mode, the event kernel's slot records
 *   opts       tracker, mode (history or event), seed, first_id, p_absorb,
 *              max_segments, queue_depth, mesh_tally (tallied in active
 *              cycles); FP64 only, no path cutoff.
 * Everything runs on `stream` without a host synchronisation (the cycle
 * count is fixed), so the whole iteration can be captured in a CUDA graph.
 * A cycle that banks no site writes TRK_E_SOURCE to counters[TRK_K_STATUS].
 * The paper's fission physics (nuclear data, energy) is out of scope: this
 * source stands in for it.
 */
trk_status power_iteration_work_bytes(trk_geom_t g, int64_t n, const trk_run_opts* opts, size_t* bytes);
trk_status power_iteration(trk_geom_t g, int64_t n, int inactive, int cycles, double* dev_k, int64_t* dev_bank,
                           uint64_t* dev_tally, uint64_t* dev_counters, void* dev_work, size_t work_bytes,
                           const trk_run_opts* opts, void* stream);

/* Bins of the description's superimposed mesh ("mesh": {"grid": [x planes,
 * y planes, z planes]}, increasing planes per axis), 0 without one.  The mesh
 * tally (trk_run_opts.mesh_tally) walks each segment across the mesh planes
 * from its start and adds each piece inside the mesh to its bin (the paper's
 * active-cycle flux tally on a superimposed mesh, Sec. 6). */
trk_status geometry_mesh_bins(trk_geom_t g, int64_t* bins);

/*
 * source_init - sample the birth state of n particles (Alg. 2: position,
 * isotropic direction, number of mean free paths tau).
 *   Position uniform over the description's source box, rejected until it
 *   lies in a root cell; direction by Marsaglia's method; tau = -log(xi).
 *   Random numbers: Philox4x32-10, key (seed_lo32, geometry id), counter
 *   ((first_id + i) mod 2^32, event 0, tag, attempt).
 *   dev_particles  caller buffer of *particle_bytes bytes (8-byte aligned),
 *                  NULL to query the size.  Layout (structure of arrays,
 *                  n entries each): double x,y,z,u,v,w,tau; int32 status.
 * Errors: TRK_E_INVALID, TRK_E_NOMEM, TRK_E_CUDA.  A particle whose source
 * sampling hit the attempt cap gets status TRK_E_SOURCE.
 */
trk_status source_init(trk_geom_t g, int64_t n, uint64_t first_id, uint64_t seed,
                       void* dev_particles, size_t* particle_bytes, void* stream);

/* Work (scratch) bytes run_histories needs for n particles with these options. */
trk_status run_histories_work_bytes(trk_geom_t g, int64_t n, const trk_run_opts* opts,
                                    size_t* bytes);

/*
 * run_histories - track n particles from their birth states to absorption,
 * escape or a cap (Alg. 2 with synthetic physics; find_cell Alg. 7,
 * cross_surface Alg. 8; distances, moves and direction changes of Table 1).
 *   dev_particles  birth states written by source_init (read only).
 *   dev_tally      uint64[n_instances], track length per leaf cell instance
 *                  in units of 2^-32 cm (added to, not cleared).
 *   dev_counters   uint64[TRK_NCOUNTERS] (added to, not cleared).
 *   dev_records    optional uint64[2n]: per particle {FNV-1a digest of the
 *                  (instance, segment-length bits) sequence,
 *                  (segments << 32) | (uint32)status}; NULL to skip.
 *   dev_work       scratch of run_histories_work_bytes (256-byte aligned).
 *   opts           NULL = defaults.
 * Errors: TRK_E_INVALID, TRK_E_UNSUPPORTED (FP32-local in the exact build,
 * FP32-local with a path cutoff), TRK_E_NOMEM, TRK_E_CUDA.
 */
trk_status run_histories(trk_geom_t g, const void* dev_particles, int64_t n, uint64_t* dev_tally,
                         uint64_t* dev_counters, uint64_t* dev_records, void* dev_work,
                         size_t work_bytes, const trk_run_opts* opts, void* stream);

/* tally_read - copy the tally to host as cm (value * 2^-32).  Synchronises
 * `stream`.  n_instances must equal the geometry's.  Also returns
 * TRK_E_TIMEOUT/TRK_E_LOST... if dev_counters (optional) holds a kernel status. */
trk_status tally_read(trk_geom_t g, const uint64_t* dev_tally, double* host_out, int64_t n_instances,
                      const uint64_t* dev_counters, void* stream);

/* trk_find_cell - Alg. 7 for n global points (dev_xyz: double[3n]); writes
 * the leaf instance or -1 (outside / lost) to dev_inst (int64[n]). */
trk_status trk_find_cell(trk_geom_t g, int tracker, int64_t n, const double* dev_xyz,
                         int64_t* dev_inst, void* stream);

/* trk_trace - run_histories (Alg. 2) that also logs each particle's
 * segments: for particle i and segment k < cap, dev_inst[i*cap+k] (int32
 * leaf instance, -1 past the end) and dev_len[i*cap+k] (segment length, cm).
 * opts->mode selects the kernel: history mode (FP64 or FP32-local), or event
 * mode, which runs the persistent event kernel in the launch shape
 * run_histories uses for the same options (tracker, precision, queue depth,
 * grid), so the logged segments are those of that kernel.  Tallies and
 * counters as in run_histories.
 *   dev_work, work_bytes  event mode: scratch of run_histories_work_bytes for
 *                         the same n and opts (256-byte aligned); history
 *                         mode: NULL, 0.
 * Errors: TRK_E_INVALID, TRK_E_NOMEM (event-mode work buffer too small),
 * TRK_E_UNSUPPORTED (FP32-local in the exact build), TRK_E_CUDA. */
trk_status trk_trace(trk_geom_t g, const void* dev_particles, int64_t n, int32_t cap,
                     int32_t* dev_inst, double* dev_len, uint64_t* dev_tally,
                     uint64_t* dev_counters, void* dev_work, size_t work_bytes,
                     const trk_run_opts* opts, void* stream);

/*
 * trk_distance_to_surface - diagnostic: for n points with directions, the
 * leaf cell by find_cell from the root (Alg. 7) and distance_to_surface
 * over its levels (Table 1), with run_histories' tie rules (smallest
 * distance; a tie goes to the top-most level, then to the first candidate
 * in the level's order).  The point is taken as on no surface.
 *   tracker    TRK_TRACKER_RECT, _CSG, _AUTO or _DP
 *   precision  TRK_FP64, or TRK_FP32_LOCAL: the distance the FP32-local
 *              flight takes (fast build; array or CSG tracker): FP32 in the
 *              level frames, a plane crossing re-evaluated in FP64, a close
 *              call (two candidates within 2e-5 relative) or an
 *              ill-conditioned cylinder redone by the FP64 scan
 *   dev_xyz    double[3n], global positions (x, y, z per point)
 *   dev_dir    double[3n], unit directions
 *   dev_dist   out double[n]: the distance in cm (+inf: no boundary ahead;
 *              NaN: the point is in no cell)
 *   dev_level  out int32[n] or NULL: level of the winning surface (-1: none)
 *   dev_inst   out int64[n] or NULL: leaf cell instance (-1: in no cell)
 *   dev_close  out int32[n] or NULL: 1 where the FP32-local distance was
 *              redone in FP64, else 0
 * Errors: TRK_E_INVALID (bad handle, null buffers, n < 0, unknown tracker or
 * precision), TRK_E_UNSUPPORTED (array tracker unavailable; FP32-local in
 * the exact build or with the DP tracker), TRK_E_CUDA.
 */
trk_status trk_distance_to_surface(trk_geom_t g, int tracker, int precision, int64_t n, const double* dev_xyz,
                                   const double* dev_dir, double* dev_dist, int32_t* dev_level, int64_t* dev_inst,
                                   int32_t* dev_close, void* stream);

/* trk_sync_status - synchronises `stream` and returns the first kernel-level
 * status a launch wrote to dev_counters[TRK_K_STATUS] (TRK_OK if none), the
 * way tally_read reports it; reads 8 bytes from the device. */
trk_status trk_sync_status(const uint64_t* dev_counters, void* stream);

/*
 * transmission_fwd - deterministic rays without collisions: per-material
 * track lengths l_m and T = exp(-sum_m sigma_m l_m) (the optical depth of
 * the track-length walk).
 *   dev_rays   double[6n] (x,y,z,u,v,w) per ray, start inside the geometry.
 *   dev_sigma  double[n_materials].
 *   dev_T      double[n]; dev_lens double[n*n_materials] (may be NULL).
 */
trk_status transmission_fwd(trk_geom_t g, int tracker, int64_t n, const double* dev_rays,
                            const double* dev_sigma, double* dev_T, double* dev_lens, void* stream);

/* Parameters of the transmission gradient beyond sigma: pin radii r_0..r_2
 * (surfaces tagged rparam) and the lattice pitch (surfaces tagged pscale). */
enum { TRK_NGEOM_PARAMS = 4 };

/* Work bytes of transmission_bwd for n rays. */
trk_status transmission_bwd_work_bytes(trk_geom_t g, int64_t n, size_t* bytes);

/*
 * transmission_bwd - hand-written backward of transmission_fwd: given
 * dL/dT per ray (dev_gT), writes dev_grad[n_materials + 4] =
 * sum_rays dL/dT * dT/dtheta for theta = (sigma_0.., r_0, r_1, r_2, pitch).
 * dT/dsigma_m = -l_m T; geometric parameters through the moved hit points:
 * dt/dtheta = -(df/dtheta)/(grad f . Omega) at every crossing, segment
 * lengths move by dt_exit - dt_entry.  Segments are recomputed, not stored.
 * The reduction over rays is a fixed-order tree (deterministic).
 */
trk_status transmission_bwd(trk_geom_t g, int tracker, int64_t n, const double* dev_rays,
                            const double* dev_sigma, double pitch, const double* dev_gT,
                            double* dev_grad, void* dev_work, size_t work_bytes, void* stream);

/*
 * Batched tracking: many independent geometries and particle populations
 * of uneven size in one persistent launch (the Alg. 2 loop over several
 * problems at once; the paper runs one problem per GPU).
 *
 * batch_create - host object over n_geom built geometries.
 *   dev_particles[k]  particle buffer of geometry k (source_init layout),
 *   counts[k]         its number of particles (<= 2^31),
 *   dev_tallies[k]    its tally (uint64[n_instances of geometry k]),
 *   dev_counters      uint64[n_geom * TRK_NCOUNTERS], geometry k at k*16,
 *   dev_records       NULL or per-geometry record arrays (as run_histories),
 *   tracker           TRK_TRACKER_AUTO, _RECT or _CSG.  AUTO: in event mode every
 *                     entry runs with the CSG tracker, in one launch; in history
 *                     mode each entry as run_histories' AUTO would.
 * Tallies and counters are added to, not cleared.  Particle ids restart at
 * first_id for every geometry (each geometry keys its own random numbers
 * with its geometry id).  The pointer arrays are host memory, read here.
 */
typedef struct trk_batch* trk_batch_t;
trk_status batch_create(const trk_geom_t* geoms, int n_geom, const void* const* dev_particles,
                        const int64_t* counts, uint64_t* const* dev_tallies, uint64_t* dev_counters,
                        uint64_t* const* dev_records, int tracker, trk_batch_t* out);
trk_status batch_destroy(trk_batch_t b);

/* Bytes of the caller-owned work buffer (256-byte aligned): the device table
 * and, for event mode, the per-geometry chunk counters and the slot records
 * of the batched event kernel's two launches at the largest queue depth
 * (512); enough for every mode and queue depth. */
trk_status batch_work_bytes(trk_batch_t b, size_t* bytes);

/* Writes the device table for chunks of `chunk` particles (0 = 512) into
 * dev_work; synchronises `stream`.  Call again to change the chunk size. */
trk_status batch_upload(trk_batch_t b, void* dev_work, size_t work_bytes, int chunk, void* stream);

/* Persistent launches over the whole batch (opts: mode, precision, block,
 * grid, queue_depth, sort_interval, max_rounds, seed, first_id, p_absorb,
 * max_segments; path cutoff ignored).  History mode: one kernel, one history per lane,
 * warps pull chunks of one geometry.  Event mode: the event kernel's queues
 * and slot records per warp, each warp working through chunks of one
 * geometry at a time: it starts on the geometry its share of the particles
 * falls in and keeps to it while it has chunks (per-geometry counters), then
 * takes the next geometry with chunks left, whose first chunk starts once the
 * warp's slots have drained; rect-tracker and CSG entries (a batch created
 * with _RECT) are two launches, the
 * CSG one on the batch's own side stream forked from `stream` by an event and
 * joined back to it (so it fills the SMs the first launch's last warps free),
 * each launch with its own slot records.  Issues memsets, kernels and that
 * fork/join on `stream` and nothing else, so after batch_upload it can be
 * captured in a CUDA graph (the fork and join become graph edges) and
 * replayed; the side stream, created at the first event-mode call, lives
 * until batch_destroy.  A kernel
 * that reaches the round limit writes TRK_E_TIMEOUT to the status counter of
 * the geometry it was on. */
trk_status run_batched(trk_batch_t b, void* dev_work, const trk_run_opts* opts, void* stream);

/* Autotuner: times block sizes {64, 96, 128} x chunk sizes {128, 512, 2048}
 * (history mode) or queue depths {384, 512} x chunk sizes {128, 256, 512,
 * 2048} x sort intervals {0, 4} (event mode, opts->mode) on the batch itself
 * (CUDA events, `reps` launches each) and writes the fastest to opts->block
 * or opts->queue_depth and opts->sort_interval, and *chunk_out, leaving the
 * table uploaded for it; *best_ms (optional) gets its time.  The trial
 * launches add to the tallies and counters: clear them afterwards.
 * Synchronises `stream`. */
trk_status batch_autotune(trk_batch_t b, void* dev_work, size_t work_bytes, trk_run_opts* opts,
                          int* chunk_out, int reps, double* best_ms, void* stream);

/*
 * transmission_bwd_noalloc - transmission_bwd for callers that cannot
 * allocate device memory themselves (for instance a program whose device
 * memory is all handed out by another framework's allocator, or a loop that
 * cannot pay for cudaMalloc's implicit synchronisation).  The paper has no
 * counterpart; it is a packaging of transmission_bwd.
 *   Same arguments as transmission_bwd minus the work buffer: the scratch
 *   (per-block partial sums) lives in a fixed 4 MiB array inside the
 *   library's device image, held on every device that loads the library.
 *   The caller still provides rays, sigma, dev_gT and dev_grad.
 *   Allocates nothing (no cudaMalloc/cudaFree, no allocating library call).
 *   The first call on a device looks up the array's address on that device;
 *   make it before any stream capture.  The address is kept for the life of
 *   the process, so the entry point must not be used on a device after
 *   cudaDeviceReset.  All calls share the array: calls whose kernels overlap
 *   on the GPU race on it.
 * Errors: TRK_E_NOMEM when n needs more scratch than the array holds (about
 * 44 million rays with 8 materials; the message gives this geometry's
 * limit), TRK_E_INVALID, TRK_E_CUDA, and those of transmission_bwd.
 */
trk_status transmission_bwd_noalloc(trk_geom_t g, int tracker, int64_t n, const double* dev_rays,
                                    const double* dev_sigma, double pitch, const double* dev_gT,
                                    double* dev_grad, void* stream);

/*
 * trk_peak_kernel - measurement support (the paper has no counterpart):
 * launches a microbenchmark of `blocks` x 256 threads on `stream` and
 * returns in *ops the number of operations it performs, for the caller to
 * divide by its CUDA-event time.
 *   kind 0  FP64 fused multiply-add chains (ops = flops, 2 per FMA)
 *   kind 1  FP32 fused multiply-add chains (ops = flops)
 *   kind 2  64-bit integer atomicAdd into nbins counters (ops = atomics)
 *   dev_scratch  caller buffer: >= 2 KB for kinds 0/1, >= 8*nbins bytes for
 *                kind 2 (its contents are overwritten).
 * Errors: TRK_E_INVALID, TRK_E_NOMEM, TRK_E_CUDA.
 */
trk_status trk_peak_kernel(int kind, int blocks, int iters, int nbins, void* dev_scratch,
                           size_t scratch_bytes, double* ops, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* TRK_H */

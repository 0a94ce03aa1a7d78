/* mm.h -- C ABI of the GB300 moving-mesh hot path (arXiv:1707.05333).
 *
 * One call sequence advances a periodic box of Voronoi cells by one step of
 * the paper's arbitrary Lagrangian-Eulerian scheme (Sec. 2):
 *   mm_tessellate     Voronoi cells of the generators by half-space clipping (Sec. 3)
 *   mm_mesh_velocity  generator velocities w = eta v + roundness correction (Sec. 4.2)
 *   mm_timestep       global CFL timestep, kept on the device (Sec. 4.2)
 *   mm_flux_step      limited gradients, half step, face reconstruction, face-frame
 *                     HLLC and the conservative charge update (Sec. 4, 4.1)
 *   mm_drift          move the generators by w dt (Sec. 2, step 5)
 * mm_step runs the whole sequence; mm_gradients exposes the gradient stage.
 *
 * Conventions for every call:
 *  - Arrays passed in are DEVICE pointers owned by the caller, struct-of-
 *    arrays, float64: positions pos[3][n] (x row, y row, z row), charges
 *    U[5][n] = (mass, momentum x,y,z, total energy) per cell, per-volume
 *    states W[5][n] = U / V, velocities w[3][n], gradients grad[15][n] with
 *    row 3*k+d holding d(W_k)/dx_d.  n >= 1 and n <= MM_MAX_CELLS.  With
 *    cfg.entropy = 1 the charges and states have a sixth row (m A and
 *    rho A, A = P / rho^gamma) and the gradients 18 rows.
 *  - Positions must lie in [0, box[d]); generators must be distinct.
 *  - Every call is enqueued on the context's stream and returns without
 *    waiting, except mm_tessellate and mm_step, which wait once for the
 *    face count and the device status word.
 *  - No call aborts.  A failure returns a nonzero mm_status and
 *    mm_last_error() describes it; device-side failures (a cell whose
 *    candidate, plane or vertex list overflowed, non-finite input) are
 *    reported by the next call that reads the status word.
 *  - Not thread-safe per context; distinct contexts are independent.
 */
#ifndef MM_H
#define MM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MM_MAX_CELLS 100000000LL /* index arithmetic is 32-bit per face/incidence */
/* Box sizes accepted by the tessellation (every axis, every box): the
 * clipper forms its bounds and limits in FP32 with explicit margins, which
 * hold while squared lengths of a few box sizes stay normal FP32 numbers.
 * Scale coordinates into this range (2^-40 .. 2^40). */
#define MM_MIN_BOX 9.094947017729282e-13
#define MM_MAX_BOX 1099511627776.0

typedef enum {
    MM_OK = 0,
    MM_EINVAL = 1,      /* bad argument, position outside the box, non-finite value */
    MM_ENOMEM = 2,      /* device allocation failed                                  */
    MM_ECAPACITY = 3,   /* a cell exceeded a fixed per-cell list even when re-clipped  */
                        /* with the large lists (see mm_tessellate)                   */
    MM_EDEGENERATE = 4, /* coincident generators, or an inconsistent mesh (near-degenerate generators) */
    MM_ECUDA = 5,       /* a CUDA runtime call failed                               */
    MM_ETIMEOUT = 6     /* reserved: a bounded device wait gave up                   */
} mm_status;

typedef struct {
    double gamma;     /* ideal-gas index: P = (gamma - 1) rho eps (Sec. 6)                  */
    double cfl;       /* eta_CFL of the per-cell timestep (Sec. 4.2)                        */
    double eta;       /* mesh velocity w = eta v; 0 static mesh, 1 Lagrangian (Sec. 4.2)    */
    double chi;       /* roundness correction speed, in sound speeds (Sec. 4.2)             */
    double zeta;      /* roundness correction radius, in effective radii (Sec. 4.2)         */
    double theta;     /* Duffell-MacFadyen limiter parameter (Sec. 4.1)                      */
    double rho_floor; /* density floor (Sec. 4.1)                                           */
    double eps_floor; /* specific internal energy floor (Sec. 4.1)                          */
    double area_rel;  /* faces with area <= area_rel (V_box/n)^(2/3) are dropped            */
    int limiter;      /* 0 none, 1 S10, 2 S10 times Duffell-MacFadyen, 3 S10 measured to   */
                      /*    face centroids (Sec. 4.1)                                       */
    int regularize;   /* 1: add the roundness correction to w (Sec. 4.2)                    */
    int precision;    /* 0: FP64 hydro; 1: mixed (FP32 gradients, half step and fluxes,     */
                      /*    FP64 update); the mesh is FP64-exact either way (clip_filter)   */
    int collect_stats;/* 1: the clipper records the counters read by mm_tess_stats          */
    int riemann;      /* 0 HLLC (the paper's default), 1 HLL (Sec. 4)                        */
    int clip_warps;   /* cells (warps) per block of the clipping kernel, 1..8 (tunable; 2)   */
    int cand_cap;     /* candidates per sorted batch of the clipper, 32..64 (tunable)        */
    int clip_filter;  /* 1: clip with FP32 vertices, an error-bounded FP32 plane test and    */
                      /*    an exact FP64 test near ties, then FP64 vertices (same mesh, bit */
                      /*    for bit); 0: solve and test every vertex in FP64 as it appears  */
    double bin_scale; /* neighbour-search bin edge in mean generator spacings (tunable)       */
    double mach_th;   /* energy/entropy switch: a cell whose largest face shock Mach number   */
                      /*    is below mach_th takes its energy from its entropy (Sec. 4.3);   */
                      /*    a face between equal states reads 0 or 1 + O(eps), so values at  */
                      /*    or below 1 let rounding decide in uniform regions (0 = energy    */
                      /*    everywhere is exact)                                              */
    int entropy;      /* 1: charges carry a sixth row m A, A = P / rho^gamma, and the switch  */
                      /*    applies (FP64 hydro only); 0: five rows, energy equation only    */
    int integrator;   /* 0: half-step predictor with start-of-step geometry (Sec. 4.1);      */
                      /*    1: Heun, fluxes averaged over start and end meshes (Sec. 6; FP64 */
                      /*    hydro, no entropy column; one more tessellation per step)        */
    int clip_sort;    /* how the clipper orders more than 32 buffered candidates: 0 in      */
                      /*    shared memory, 1 in registers (same order and mesh; tunable)      */
} mm_config;

/* Fill a config with the defaults: gamma 5/3, cfl 0.3, eta 1, chi 1, zeta
 * 0.25, theta 0.49, floors 1e-10, area_rel 1e-10, S10 limiter, no
 * roundness correction, FP64 hydro, filtered clipping, no counters, HLLC,
 * 2 clip warps per block, batches of 64 candidates, bins one mean spacing
 * wide, no entropy column (mach_th 1.1 when it is switched on), half-step
 * time integration, candidates over 32 sorted in shared memory. */
void mm_default_config(mm_config *cfg);

typedef struct mm_ctx mm_ctx;

/* The mesh of the last mm_tessellate: DEVICE pointers owned by the context,
 * valid until the next mm_tessellate / mm_step or mm_destroy.
 * Faces are unique: face f joins cells face_i[f] and face_j[f], where the
 * neighbour sits at its periodic image pos_j + s L with s decoded from
 * face_shift[f] = (sx+1) + 3 (sy+1) + 9 (sz+1); face_i < face_j, or
 * face_i == face_j with face_shift > 13 (a cell touching its own image).
 * face_normal is the unit vector from i towards j's image; face_centroid is
 * in cell i's frame (add -s L for j's).  Cell k's faces are
 * inc_face[inc_off[k] .. inc_off[k+1]); an entry f >= 0 means k is face_i[f]
 * (outward normal +n), an entry ~f (< 0) means k is face_j[f] (normal -n).
 * cell_centroid is r_k + (centroid relative to r_k): it may lie outside the
 * box near the boundary.  A batched mesh (mm_step_batched) holds nboxes
 * independent boxes; every dt argument below is then one value per box. */
typedef struct {
    int64_t n, nfaces, nincident;
    int64_t face_stride; /* row stride of face_normal and face_centroid (>= nfaces) */
    double box[3];       /* size of box 0 (the only box of a single-box mesh) */
    int64_t nboxes;      /* independent periodic boxes stored back to back */
    const int32_t *cell_box; /* [n] box of each cell */
    const double *box_size;  /* [nboxes][3] box sizes */
    const int32_t *face_i, *face_j, *face_shift;
    const double *face_area;     /* [F]    */
    const double *face_normal;   /* [3][face_stride] */
    const double *face_centroid; /* [3][face_stride] */
    const double *cell_volume;   /* [n]    */
    const double *cell_centroid; /* [3][n] */
    const int32_t *inc_off;      /* [n+1]  */
    const int32_t *inc_face;     /* [nincident] */
} mm_mesh;

/* Create a context whose work runs on `cuda_stream` (a cudaStream_t, or NULL
 * for the legacy default stream) of the current device.  The context owns
 * its device workspace and grows it on demand. */
mm_status mm_create(mm_ctx **ctx, const mm_config *cfg, void *cuda_stream);
void mm_destroy(mm_ctx *ctx);
const char *mm_last_error(const mm_ctx *ctx);
mm_status mm_set_config(mm_ctx *ctx, const mm_config *cfg);

/* Voronoi tessellation of the periodic box [0,box) (Sec. 3).  Each cell
 * starts as the box centred on its generator (whose six faces are the
 * bisectors with the generator's own images) and is clipped by the
 * bisector planes of neighbouring generators and images in increasing
 * distance, until every remaining generator is more than twice as far as
 * the farthest vertex.  pos[3][n] device.  Box sizes outside
 * [MM_MIN_BOX, MM_MAX_BOX] are MM_EINVAL (here, in mm_step, mm_step_batched
 * and mm_autotune).  Waits for completion.
 * Capacities: a cell is first clipped with lists of 64 planes, 128 vertices,
 * 32 new vertices per cut, 48 faces and 48 search rings; a cell that
 * overflows one is clipped again by a large instance of the clipper (128
 * planes, 256 vertices, 64 new vertices per cut, 128 faces, 128 rings)
 * whose faces go to an overflow row of that cell.  Only a cell beyond the
 * large lists fails the call with MM_ECAPACITY.  Overflow rows are grown to
 * the number of such cells here; a captured batch (mm_step_batched) has 256
 * and reports more through mm_sync_status.  Two generators at the same
 * position (or at the same periodic image) are MM_EDEGENERATE.
 * Ties: a vertex lies beyond a plane only past a margin of 2^-40..2^-39 of
 * the plane's offset, so generators on exact lattices (cubic, bcc, fcc:
 * several cells sharing each vertex) tessellate; a cell whose cut is
 * inconsistent under that margin is clipped again with the strict rule.
 * A cell inconsistent under both, or two cells that disagree on a face far
 * above the area threshold (1e4 times it), make the call MM_EDEGENERATE
 * rather than return such a mesh (seen for cubic lattices perturbed by
 * 1e-13..1e-11 of a spacing and for generators 1e-10 apart). */
mm_status mm_tessellate(mm_ctx *ctx, const double *pos, int64_t n, const double box[3], mm_mesh *out);

/* Limited cell-centred gradient of per-volume states W[5][n] (Sec. 4.1):
 * grad W_i = M_i^-1 b_i with M_i = 1/2 sum_j A n (x) (c_j - c_i) and
 * b_i = 1/2 sum_j A (W_j - W_i) n, then the S10 factor min(1, psi_ij) and,
 * for limiter 2, the Duffell-MacFadyen factor min(1, max(0, theta (W_j -
 * W_i) / Delta_ij)) over the neighbours whose Delta_ij = grad W_i . (c_j -
 * c_i) exceeds 2^-40 |grad W_i|_1 |c_j - c_i|_1 in size (below that it is
 * zero up to rounding, as toward the equal-valued transverse neighbours of
 * a lattice with a planar state).  grad[15][n] device.  The
 * context forms the per-face A n and separations in its own workspace
 * (grown on demand, like the other stages'). */
mm_status mm_gradients(mm_ctx *ctx, const mm_mesh *mesh, const double *W, double *grad);

/* w = eta v (+ chi c_s d/|d| ramp(|d| / zeta R) when regularize) (Sec. 4.2).
 * pos[3][n], U[5][n] in; w[3][n] out. */
mm_status mm_mesh_velocity(mm_ctx *ctx, const mm_mesh *mesh, const double *pos, const double *U,
                           double *w);

/* dt = min_i cfl R_i / (c_s,i + |v_i - w_i|), written to the device scalar
 * *dt (Sec. 4.2). */
mm_status mm_timestep(mm_ctx *ctx, const mm_mesh *mesh, const double *U, const double *w, double *dt);

/* One conservative update of the charges U[5][n] (in place) over the mesh:
 * gradient of W^n, half step W^(n+1/2) = W^n - dt/2 sum_d A_d dW/dx_d, its
 * gradient, reconstruction to face centroids, floors, boost into the frame
 * of each moving face, HLLC, boost back, and U_i -= dt sum_faces (+-) A F
 * (Sec. 4, 4.1).  With cfg.entropy the sixth row is advected as a passive
 * scalar and each cell keeps the energy equation only where its largest face
 * shock Mach number reaches cfg.mach_th, else takes E from its entropy
 * (Sec. 4.3).  dt is a DEVICE pointer to one double (e.g. from
 * mm_timestep).  pos[3][n] are the generator positions the mesh was built
 * from; w[3][n] the generator velocities. */
mm_status mm_flux_step(mm_ctx *ctx, const mm_mesh *mesh, const double *pos, const double *w,
                       const double *dt, double *U);

/* pos += w dt, wrapped into [0, box) (Sec. 2, step 5).  dt device scalar. */
mm_status mm_drift(mm_ctx *ctx, double *pos, int64_t n, const double *w, const double *dt,
                   const double box[3]);

/* One whole step in place: tessellate pos, w = mesh velocity, dt = CFL
 * timestep (or *dt_fixed when dt_fixed != NULL, a device scalar), flux step
 * on U, drift pos.  dt_out (device scalar, may be NULL) receives dt and
 * w_out (device [3][n], may be NULL) receives w. */
mm_status mm_step(mm_ctx *ctx, double *pos, double *U, int64_t n, const double box[3],
                  const double *dt_fixed, double *dt_out, double *w_out);

/* One whole step (as mm_step, CFL timestep) on HOST arrays: pos[3][n] and
 * U[5][n] (U[6][n] with cfg.entropy) are read from host memory and
 * overwritten with the step's result; dt_out (host, may be NULL) receives
 * dt.  The context keeps device copies (grown as needed, freed by
 * mm_destroy).  The copies overlap the step: the positions go up first (the
 * binning reads them), the charges on a second stream while the mesh is
 * built (the mesh velocity reads them first), and the new charges come back
 * while the generators drift.  With page-locked host memory (cudaHostAlloc,
 * torch pin_memory) the copies are asynchronous; pageable memory works but
 * serialises them.  Returns once the results are in the host arrays.  The
 * caller keeps ownership of the host arrays. */
mm_status mm_step_host(mm_ctx *ctx, double *pos, double *U, int64_t n, const double box[3], double *dt_out);

/* One whole step (as mm_step, CFL timestep per box) for nboxes independent
 * periodic boxes stored back to back: box b holds cells
 * [box_off[b], box_off[b+1]) of pos[3][n] and U[5][n] and has size
 * boxes[3b..3b+2]; box_off and boxes are HOST arrays, box_off[0] = 0 and
 * box_off[nboxes] = n.  Every box is an independent problem: its own bins,
 * face threshold and timestep; results equal mm_step on each box alone.
 * The first call for a given (pos, U, n, boxes, dt_out, config) reserves
 * fixed capacities (10 n unique faces), captures the whole step into a CUDA
 * graph on the context's stream (which must not be the legacy default
 * stream) and launches it; later identical calls only relaunch the graph,
 * with no host synchronisation.  dt_out (device [nboxes], may be NULL)
 * receives each box's dt.  Device-side failures (including a capacity
 * overflow) are reported by mm_sync_status. */
mm_status mm_step_batched(mm_ctx *ctx, double *pos, double *U, int64_t n, const int64_t *box_off,
                          const double *boxes, int nboxes, double *dt_out);

/* The context's current configuration. */
mm_status mm_get_config(const mm_ctx *ctx, mm_config *cfg);

/* Pick clip_warps, cand_cap, bin_scale and clip_sort for generators like
 * pos[3][n] in box: every combination of {2,4,8} x {32,64} x
 * {0.8,1,1.25,1.5} x {0,1} is timed on
 * `reps` tessellations (after one warm-up each) and the fastest is kept in
 * the context's configuration; *best_ms (may be NULL) receives its time.
 * The mesh of the last timed tessellation is left in the context. */
mm_status mm_autotune(mm_ctx *ctx, const double *pos, int64_t n, const double box[3], int reps, double *best_ms);

/* Wait for the context's stream and report the device status word of the
 * last tessellation (mm_step_batched does not wait on its own). */
mm_status mm_sync_status(mm_ctx *ctx);

/* The mesh of the last tessellation (waits; for a batched step the face and
 * incidence counts are read back from the device). */
mm_status mm_current_mesh(mm_ctx *ctx, mm_mesh *out);

/* Charges from per-volume primitives on the current mesh:
 * U = (rho, rho v, P/(gamma-1) + rho |v|^2 / 2) V, and with cfg.entropy the
 * sixth row rho V P / rho^gamma.  rho[n], vel[3][n], P[n]. */
mm_status mm_prims_to_charges(mm_ctx *ctx, const mm_mesh *mesh, const double *rho, const double *vel,
                              const double *P, double *U);

/* Per-component totals of U[5][n] as compensated (Neumaier) FP64 sums,
 * written to the device array totals[5]. */
mm_status mm_totals(mm_ctx *ctx, const double *U, int64_t n, double *totals);

/* Per-component totals of U[5][n] like mm_totals, for callers that cannot
 * allocate device memory: code running while a stream is captured into a
 * CUDA graph (no cudaMalloc there), code that must not synchronise the device
 * (cudaFree does), and hosts whose own pool owns all device memory.  It needs
 * no context and allocates nothing: its scratch is a fixed array of 320 KiB
 * inside this library's device image, placed on a device when the library is
 * loaded there and held until the process exits.  The paper has no
 * counterpart; this is a service entry point of the library.
 *  - U[5][n] and totals[5] are device pointers owned by the caller; work is
 *    enqueued on cuda_stream (a cudaStream_t, or NULL) without waiting.
 *  - n must be in [1, MM_TOTALS_NOALLOC_MAX_CELLS]; a larger n returns
 *    MM_ECAPACITY, n < 1 or a NULL pointer MM_EINVAL.  When err is not NULL,
 *    a message of at most err_len bytes (NUL-terminated) describes a failure.
 *  - The first call on a device looks up the scratch array's device address
 *    (once per device, with that device current); make that first call
 *    before any stream capture.
 *  - Every call shares the one scratch array, which keeps the last call's
 *    partial sums; each call writes every partial it reads, so nothing has to
 *    start at zero.  Calls whose kernels overlap on the GPU (other streams,
 *    other threads) race on the scratch and give wrong totals: order them.
 *  - Results agree with mm_totals to rounding (compensated sums over tiles of
 *    4096 cells instead of the context's fixed block ranges). */
#define MM_TOTALS_NOALLOC_MAX_CELLS 16777216LL
mm_status mm_totals_noalloc(const double *U, int64_t n, double *totals, void *cuda_stream, char *err,
                            int64_t err_len);

/* Stream-ordered device-to-device copy of `bytes` bytes (a convenience for
 * bindings that read the context-owned mesh arrays into their own buffers). */
mm_status mm_copy(mm_ctx *ctx, void *dst, const void *src, int64_t bytes);

/* Device-side counters of the last tessellation made with
 * mm_config.collect_stats = 1, copied to the host:
 * [0] max candidates in one sorted batch, [1] max planes of a cell,
 * [2] max vertices of a cell, [3] cells needing more than one search ring,
 * [4] total cuts, [5] FP64 plane tests, [6] FP64 three-plane solves,
 * [7] FP64 face-fan terms, [8] candidates tested, [9] cells re-clipped by the
 * large-capacity clipper (counted with or without collect_stats). */
#define MM_NSTATS 10
mm_status mm_tess_stats(mm_ctx *ctx, int64_t stats[MM_NSTATS]);

/* Stages of a step, for per-stage device timing. */
typedef enum {
    MM_STAGE_BIN = 0,           /* generator binning (neighbour search structure)   */
    MM_STAGE_CLIP = 1,          /* per-cell clipping                                */
    MM_STAGE_FACES = 2,         /* face confirmation, scans, unique faces, CSR      */
    MM_STAGE_MESH_VELOCITY = 3, /* mesh velocity and CFL timestep                   */
    MM_STAGE_GRADIENT_HALF = 4, /* limited gradient of W^n fused with the half step */
    MM_STAGE_GRADIENT = 5,      /* limited gradient of W^(n+1/2)                    */
    MM_STAGE_FACE_FLUX = 6,     /* reconstruction, face-frame HLLC, back-boost      */
    MM_STAGE_UPDATE = 7,        /* conservative charge update                       */
    MM_STAGE_DRIFT = 8,         /* generator drift                                  */
    MM_NSTAGES = 9
} mm_stage;

/* on != 0: from now on record CUDA events around every stage on the
 * context's stream (a few microseconds of host work per stage); resets the
 * accumulated times.  on == 0 stops recording. */
mm_status mm_set_timing(mm_ctx *ctx, int on);

/* Wait for the stream, then return the summed device time in ms of each
 * stage since mm_set_timing, and how many times each stage ran. */
mm_status mm_stage_times(mm_ctx *ctx, double ms[MM_NSTAGES], int64_t runs[MM_NSTAGES]);

/* Number of kernels this context has launched since it was created. */
int64_t mm_kernel_launches(const mm_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif

/*
 * ibip.h -- C ABI of libibip: image-based invasion percolation (IBIP) on one
 * NVIDIA GB300 GPU.
 *
 * The method: Gostick, Yang & Boek, "Simulating volume-controlled invasion of
 * a non-wetting fluid in volumetric images using basic image processing
 * tools", arXiv 2101.03240.  Section numbers below refer to that paper.
 *
 * Conventions shared by every call
 *   - A voxel image has shape (nx, ny, nz) in C order: the linear index of
 *     voxel (x, y, z) is idx = (x*ny + y)*nz + z, so z is contiguous.
 *   - uint8 images: nonzero = pore (void), 0 = solid.  Connectivity is 6
 *     (face neighbours) everywhere.  Voxels outside the image are not solid.
 *   - dt2 (int32): squared Euclidean distance from a pore voxel to the
 *     nearest solid voxel; 0 on solid; INT32_MAX on pore when the image holds
 *     no solid voxel at all.
 *   - seq (int32): 0 solid, -1 pore never invaded (or reset by trapping),
 *     k >= 1 invaded at step k.
 *   - Every dimension must be in [1, 16384] and nx*ny*nz < 2^31.
 *
 * Memory, streams and errors
 *   - Array arguments are DEVICE pointers on the context's device unless the
 *     name starts with h_ (host memory).  The caller owns every argument
 *     buffer; the context owns its scratch memory and reuses it across calls.
 *   - Work is queued on the context's stream.  Calls that return a value
 *     through an h_ pointer synchronise that stream before returning; the
 *     others return as soon as the work is queued.
 *   - Arguments are validated on the host before any launch; a bad argument
 *     returns IBIP_ERR_ARG and queues nothing.  Limits reached on the device
 *     (step limit, round limit) are reported by the synchronising calls.
 *     Results are unspecified after any status other than IBIP_OK, except
 *     where a call documents otherwise.
 *   - No C++ exception crosses this interface.  A context is not thread-safe;
 *     use one context per host thread.
 */
#ifndef IBIP_H
#define IBIP_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define IBIP_API __attribute__((visibility("default")))
#else
#define IBIP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    IBIP_OK = 0,
    IBIP_ERR_ARG = -1,           /* invalid argument (nothing queued) */
    IBIP_ERR_CUDA = -2,          /* a CUDA runtime call failed */
    IBIP_ERR_OOM = -3,           /* scratch allocation failed */
    IBIP_ERR_STEP_LIMIT = -4,    /* invasion stopped at max_steps with candidates left */
    IBIP_ERR_NOT_CONVERGED = -5, /* propagation hit its round or activation limit, or stalled */
    IBIP_ERR_CANCELLED = -6,     /* the invasion stopped at a cancel request (ibip_cancel) */
    IBIP_ERR_BOUNDS = -7,        /* a device-side index check failed (progress guard; any
                                    index of the invasion loop in a build with IBIP_CHECKED) */
    IBIP_ERR_TOO_LARGE = -8      /* image larger than ibip_edt_noalloc's fixed scratch */
} ibip_status;

/* Image faces: X0 is the face x = 0, X1 is x = nx-1, and so on. */
typedef enum { IBIP_X0 = 0, IBIP_X1, IBIP_Y0, IBIP_Y1, IBIP_Z0, IBIP_Z1 } ibip_face;

typedef struct { int32_t nx, ny, nz; } ibip_dims;

typedef struct ibip_ctx ibip_ctx;

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * to queue work on (the caller keeps owning it), or NULL: the context then
 * creates a non-blocking stream of its own, which it destroys in
 * ibip_destroy, so that its work never serialises against unrelated work on
 * the legacy default stream.  To queue on the legacy default stream itself,
 * pass cudaStreamLegacy ((void *)0x1); cudaStreamPerThread ((void *)0x2)
 * works the same way.  Writes the new context to *out.  Returns IBIP_OK,
 * IBIP_ERR_ARG or IBIP_ERR_CUDA. */
IBIP_API int ibip_create(ibip_ctx **out, int device, void *cuda_stream);

/* Release the context, its scratch memory and its own stream (if it has
 * one); synchronises the streams first. */
IBIP_API int ibip_destroy(ibip_ctx *ctx);

/* Change the stream later calls queue on: a cudaStream_t (cudaStreamLegacy
 * for the legacy default stream), or NULL for the context's own
 * non-blocking stream (created here if the context has none yet).  Work
 * queued earlier is not waited for: order the two streams yourself. */
IBIP_API int ibip_set_stream(ibip_ctx *ctx, void *cuda_stream);

/* The stream calls currently queue on (*h_stream; never NULL: the legacy
 * default stream reads as cudaStreamLegacy only if it was given as such). */
IBIP_API int ibip_get_stream(const ibip_ctx *ctx, void **h_stream);

/* Whether this context's kernels may run beside long-running kernels of
 * other streams or contexts on the same device (on != 0), for instance an
 * invasion running on another stream while this context computes the
 * opening.  The widest-path propagation (trapping, the opening's trim) then
 * runs one ordinary launch per round, the host reading the next round's
 * list size every 16 rounds, so that the other streams' blocks get in
 * between rounds.  It never runs as one cooperative grid, whose blocks must
 * all be resident at once, nor on its work queue, whose resident blocks
 * would hold the SMs until the propagation ends; those serve a context
 * that has the device to itself.  Results are the same every way.  Default
 * off; server slots always run this way.  IBIP_ERR_ARG for a NULL ctx. */
IBIP_API int ibip_set_shared_device(ibip_ctx *ctx, int on);

/* Squared Euclidean distance transform of the pore space (Section 2.1,
 * Figure 2b).
 *   image: uint8[nx*ny*nz], nonzero = pore.
 *   dt2:   int32[nx*ny*nz] output as defined above (exact integers).
 * Asynchronous. */
IBIP_API int ibip_edt(ibip_ctx *ctx, const uint8_t *image, ibip_dims dims, int32_t *dt2);

/* ibip_edt without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that must not allocate device memory
 * at call time -- code whose device memory is owned by a pool, an arena or a
 * host framework that forbids (or would be fragmented by) direct cudaMalloc,
 * and latency-sensitive loops that cannot afford the implicit device-wide
 * synchronisation cudaMalloc/cudaFree may cause.  It takes no context.
 *   image:       uint8[nx*ny*nz] device buffer, nonzero = pore.
 *   dims:        nx*ny*nz must not exceed 2^21 (2,097,152) voxels, e.g. 128^3;
 *                larger images return IBIP_ERR_TOO_LARGE and queue nothing.
 *   dt2:         int32[nx*ny*nz] device output, same values as ibip_edt.
 *                Its memory also holds an intermediate during the call.
 *   cuda_stream: cudaStream_t to queue on (NULL = legacy default stream).
 * Works on the current CUDA device.  Scratch is one fixed 8 MB device array
 * compiled into the library: every GPU that loads the library keeps it until
 * the process exits, and every call on a device shares it, so calls that
 * overlap on the GPU (other streams, other host threads) race and must be
 * serialised by the caller.  The first call on each device looks up that
 * array's device address once; make that first call before any stream
 * capture on the device.  Allocates nothing: no cudaMalloc, no cudaFree.
 * Asynchronous.  Returns IBIP_OK, IBIP_ERR_ARG, IBIP_ERR_TOO_LARGE or
 * IBIP_ERR_CUDA. */
IBIP_API int ibip_edt_noalloc(const uint8_t *image, ibip_dims dims, int32_t *dt2, void *cuda_stream);

/* Volume-controlled invasion (Section 2.1, Figures 1-2; footnote 1).
 * Step k = 1, 2, ... picks the candidate voxel c with the largest dt2 --
 * candidates are uninvaded pore voxels that are 6-adjacent to an invaded
 * voxel or lie on the `inlet` face -- with ties going to the lowest linear
 * index, then writes k into every uninvaded voxel p with |p - c|^2 < dt2[c]
 * (never overwriting an earlier step).  Stops when no candidate is left or
 * after max_steps steps.
 *   image:       uint8[N] pore image.
 *   dt2:         int32[N] squared EDT of `image`, or NULL to compute it here
 *                (into context scratch).  Must be consistent with `image`.
 *   inlet:       ibip_face the non-wetting phase enters through.
 *   max_steps:   >= 0; the step limit.
 *   seq:         int32[N] output sequence image.
 *   step_r2:     int32[capacity_steps] output: dt2 of each step's centre.
 *   step_centre: int32[capacity_steps] output: linear index of each centre,
 *                or NULL.
 *   capacity_steps: length of the step arrays.
 *   h_n_steps:   host int64 output: number of steps K taken.
 * Synchronous.  Returns IBIP_ERR_STEP_LIMIT when max_steps stopped the run
 * with candidates left (seq and the step arrays hold the first max_steps
 * steps), and IBIP_ERR_ARG with *h_n_steps = K when K > capacity_steps (seq
 * is complete; only the first capacity_steps step entries are written).
 * capacity_steps = number of pore voxels is always enough. */
IBIP_API int ibip_invade(ibip_ctx *ctx, const uint8_t *image, const int32_t *dt2, ibip_dims dims,
                int inlet, int64_t max_steps, int32_t *seq, int32_t *step_r2,
                int32_t *step_centre, int64_t capacity_steps, int64_t *h_n_steps);

/* ibip_invade with two extensions of Section 2.1.
 *   inlet_mask: uint8[N] or NULL.  Nonzero voxels are the inlets (Section
 *               2.1 marks inlets with a Boolean image; they may lie inside
 *               the image, e.g. for evaporation): the pore
 *               voxels among them are the first candidates.  NULL: the
 *               `inlet` face, as ibip_invade.
 *   resume:     0, or 1 to continue an earlier run: seq then holds on entry
 *               the sequence image an earlier call wrote (steps 1..K0, where
 *               K0 is its largest value; -1 uninvaded pore; 0 solid) for the
 *               same image and inlets, and step_r2 / step_centre hold its
 *               first K0 entries.  The candidates are rebuilt from seq (inlet
 *               voxels and neighbours of invaded voxels that are still
 *               uninvaded), steps K0+1, ... are appended, and max_steps counts
 *               the new steps only.  The result equals one uninterrupted run.
 *   h_n_steps:  the total K.
 * Other arguments, statuses and synchronisation as ibip_invade. */
IBIP_API int ibip_invade_ex(ibip_ctx *ctx, const uint8_t *image, const int32_t *dt2, ibip_dims dims, int inlet,
                            const uint8_t *inlet_mask, int resume, int64_t max_steps, int32_t *seq,
                            int32_t *step_r2, int32_t *step_centre, int64_t capacity_steps, int64_t *h_n_steps);

/* The invasion exactly as Section 2.1 prints it (the "paper-literal" rule;
 * ibip_invade uses the frontier rule instead).  The inlets start as every
 * voxel of the `inlet` face.  Step k = 1, 2, ...: the candidates are the
 * inlets plus their face neighbours; every candidate holding the largest
 * dt2 is an insertion point of step k (all tied maxima at once); around each
 * one, every pore voxel p with |p - c|^2 <= R^2, R = floor(sqrt(dt2)) (the
 * truncated integer radius of footnote 1), that no earlier step invaded
 * gets k; the insertion points then join the inlets and their value is set
 * to zero.  Stops when the largest candidate value is zero, or after
 * max_steps steps.
 *   image, dt2, dims, inlet, max_steps, seq: as in ibip_invade.
 *   cstep:       int32[N] output: the step at which each voxel was an
 *                insertion point, 0 if never.
 *   step_r2:     int32[capacity_steps] output: R^2 of each step.
 *   step_count:  int32[capacity_steps] output: insertion points of each step.
 *   h_n_steps:   host int64 output: steps K.
 * Synchronous.  Status conventions as ibip_invade (capacity_steps = number
 * of pore voxels is always enough). */
IBIP_API int ibip_invade_literal(ibip_ctx *ctx, const uint8_t *image, const int32_t *dt2, ibip_dims dims,
                                 int inlet, int64_t max_steps, int32_t *seq, int32_t *cstep, int32_t *step_r2,
                                 int32_t *step_count, int64_t capacity_steps, int64_t *h_n_steps);

/* Defending-phase trapping (Section 2.2.3).  A voxel invaded at step k is
 * trapped when no 6-path through pore voxels whose sequence value is >= k
 * (never-invaded pore counting as +infinity) joins it to a pore voxel on the
 * `outlet` face.  Never-invaded voxels are not reported as trapped;
 * outlet-face voxels never are.
 *   seq:      int32[N] sequence image (from ibip_invade).
 *   outlet:   ibip_face.
 *   rerank:   nonzero to re-rank seq_out's surviving step values to
 *             1..K' in order (Section 2.2.3, contiguous sequence).
 *   trapped:  uint8[N] output, 1 = trapped.
 *   seq_out:  int32[N] output (seq with trapped voxels set to -1), or NULL.
 * Synchronous (the propagation loop checks convergence on the host);
 * returns IBIP_ERR_NOT_CONVERGED if the round limit was reached. */
IBIP_API int ibip_trapping(ibip_ctx *ctx, const int32_t *seq, ibip_dims dims, int outlet, int rerank,
                  uint8_t *trapped, int32_t *seq_out);

/* Trapping with re-ranking (Section 2.2.3) that also re-indexes the step
 * radii, so the re-ranked sequence feeds ibip_pc_curve directly.  Steps
 * left without any voxel after trapping are dropped and the survivors are
 * numbered 1, 2, ... in their old order.
 *   seq, dims, outlet, trapped: as ibip_trapping; seq_out: required.
 *   step_r2:       int32[n_steps] radii of the original steps.
 *   step_r2_out:   int32[n_steps] output: radii of the surviving steps.
 *   h_n_steps_out: host int64 output: number of surviving steps.
 * Synchronous. */
IBIP_API int ibip_trapping_ex(ibip_ctx *ctx, const int32_t *seq, ibip_dims dims, int outlet, uint8_t *trapped,
                              int32_t *seq_out, const int32_t *step_r2, int64_t n_steps, int32_t *step_r2_out,
                              int64_t *h_n_steps_out);

/* Sphere-size image (Section 2.2.2, Figure 5 right): r2_image[v] =
 * step_r2[seq[v] - 1] for 1 <= seq[v] <= n_steps (the squared radius of the
 * sphere that invaded v), 0 on solid, -1 on uninvaded pore.  Asynchronous. */
IBIP_API int ibip_size_image(ibip_ctx *ctx, const int32_t *seq, ibip_dims dims, const int32_t *step_r2,
                             int64_t n_steps, int32_t *r2_image);

/* Pressure-based drainage by morphological image opening, MIO (Section 1,
 * Section 2.4.1): for each squared radius T_i (strictly decreasing), keep
 * the pore voxels with dt2 >= T_i (erosion), trim those not 6-connected
 * inside that set to the inlet face (after the erosion, before the
 * dilation), then dilate by the ball d^2 < T_i.
 *   image, dt2:  as for ibip_invade (dt2 required).
 *   h_r2_levels: host int32[n_levels], strictly decreasing, >= 1;
 *                0 <= n_levels <= 8192.
 *   level:       int32[N] output: i+1 for the first level i that invades the
 *                voxel, -1 pore never invaded, 0 solid.
 *   h_counts:    host int64[n_levels] output: voxels with 1 <= level <= i+1.
 * Synchronous. */
IBIP_API int ibip_morph_drainage(ibip_ctx *ctx, const uint8_t *image, const int32_t *dt2, ibip_dims dims,
                        int inlet, const int32_t *h_r2_levels, int32_t n_levels, int32_t *level,
                        int64_t *h_counts);

/* ibip_morph_drainage with the dilation's bound given separately: level i
 * erodes to dt2 >= h_r2_levels[i] and dilates by the ball
 * d^2 < h_dilate_r2[i] (host int32[n_levels], each >= 1; NULL = the same
 * bounds as the erosion, i.e. ibip_morph_drainage).  With h_r2_levels[i] =
 * R^2 and h_dilate_r2[i] = R^2 + 1 for integer radii R the structuring
 * element is the closed ball |d|^2 <= R^2 of the paper-literal invasion
 * (Section 2.1, footnote 1: integer radius; ibip_invade_literal), so the
 * two can be compared at equal saturation with the element held fixed
 * (Section 3.1.1).  Other arguments, errors and synchronisation as
 * ibip_morph_drainage. */
IBIP_API int ibip_morph_drainage_ex(ibip_ctx *ctx, const uint8_t *image, const int32_t *dt2, ibip_dims dims,
                                   int inlet, const int32_t *h_r2_levels, const int32_t *h_dilate_r2,
                                   int32_t n_levels, int32_t *level, int64_t *h_counts);

/* Equal-saturation comparison of an invasion with morphological-opening
 * drainage (Section 3.1.1, Figure 8), by integer counts.  For opening level
 * i (0-based): n_i = voxels with 1 <= level <= i + 1; k_i = the smallest
 * step with #(1 <= seq <= k_i) >= n_i (n_steps if none); diff_i = the number
 * of voxels in exactly one of {1 <= level <= i + 1} and {1 <= seq <= k_i}.
 *   seq:      int32[N] sequence image (ibip_invade, ibip_invade_literal, or a
 *             trapping-corrected seq_out); values above n_steps are ignored.
 *   level:    int32[N] from ibip_morph_drainage (-1 none, 0 solid, i + 1).
 *   n_levels: 1..254.
 *   h_steps, h_count: host int64[n_levels] outputs k_i and n_i, or NULL.
 *   h_diff:   host int64[n_levels] output diff_i.
 * Synchronous. */
IBIP_API int ibip_equal_saturation(ibip_ctx *ctx, const int32_t *seq, const int32_t *level, ibip_dims dims,
                                   int64_t n_steps, int32_t n_levels, int64_t *h_steps, int64_t *h_diff,
                                   int64_t *h_count);

/* Saturation and capillary pressure after each step (Sections 2.2.1 and
 * 2.2.2; Washburn relation Pc = -2 sigma cos(theta) / R, Section 2.4.1).
 *   S_k  = (voxels with 1 <= seq <= k) / (all pore voxels, seq != 0);
 *   Pc_k = (-2 sigma cos(theta)) / (sqrt(step_r2[k]) * voxel_m), with
 *          cos(theta) = cos(theta_deg * pi / 180); double precision, one
 *          rounding to float.
 *   seq:          int32[N] (seq or a trapping-corrected seq_out).
 *   step_r2:      int32[n_steps].
 *   sat_per_step, pc_per_step: float[n_steps] outputs.
 *   sat_image:    float[N] output or NULL: S_{seq[v]} where 1 <= seq[v] <=
 *                 n_steps, +infinity elsewhere (Section 2.2.1: thresholding
 *                 it at s gives the configuration at saturation s).
 * Asynchronous. */
IBIP_API int ibip_pc_curve(ibip_ctx *ctx, const int32_t *seq, ibip_dims dims, const int32_t *step_r2,
                  int64_t n_steps, double voxel_m, double sigma, double theta_deg,
                  float *sat_per_step, float *pc_per_step, float *sat_image);

/* Drainage envelope of an invasion at the pressures of opening levels
 * (Section 2.2.2: the envelope of the invasion's peak pressures; Section
 * 3.1.1: it matches the opening's capillary-pressure curve).  Pc falls as
 * the sphere grows, so the running peak of Pc up to step k is the Pc of the
 * smallest step_r2 so far; at the pressure of level i (squared radius
 * h_r2_levels[i]) the invasion has taken every step before its running
 * minimum of step_r2 first drops below h_r2_levels[i].
 *   seq:          int32[N] sequence image (or a trapping-corrected seq_out).
 *   step_r2:      int32[n_steps].
 *   h_r2_levels:  host int32[n_levels], strictly decreasing, >= 1;
 *                 1 <= n_levels <= 254.
 *   h_steps:      host int64[n_levels] output: the number of steps taken at
 *                 level i (the first step below it, 0-based; n_steps if none).
 *   h_count:      host int64[n_levels] output: voxels with 1 <= seq <=
 *                 h_steps[i], to compare with ibip_morph_drainage's counts.
 * Synchronous. */
IBIP_API int ibip_pc_envelope(ibip_ctx *ctx, const int32_t *seq, ibip_dims dims, const int32_t *step_r2,
                              int64_t n_steps, const int32_t *h_r2_levels, int32_t n_levels, int64_t *h_steps,
                              int64_t *h_count);

/* One image of a batched call.  Device pointers unless stated; the caller
 * owns every buffer.  Outputs are those of ibip_edt, ibip_invade,
 * ibip_trapping and ibip_pc_curve for this image. */
typedef struct {
    const uint8_t *image;     /* uint8[N] pore image */
    ibip_dims dims;
    int32_t inlet;            /* ibip_face */
    int32_t outlet;           /* ibip_face for trapping, or -1 for none */
    int32_t *dt2;             /* int32[N] output, or NULL (kept in scratch) */
    int32_t *seq;             /* int32[N] output */
    int32_t *step_r2;         /* int32[capacity_steps] output */
    int32_t *step_centre;     /* int32[capacity_steps] output, or NULL */
    int64_t capacity_steps;   /* >= number of pore voxels is always enough */
    uint8_t *trapped;         /* uint8[N] output, or NULL: no trapping */
    int32_t *seq_out;         /* int32[N] output (trapped voxels -1), or NULL */
    float *sat_per_step;      /* float[capacity_steps] output, or NULL: no curve */
    float *pc_per_step;       /* float[capacity_steps] output, or NULL */
    double voxel_m, sigma, theta_deg;   /* Pc parameters (Section 2.2.2) */
    int64_t n_steps;          /* filled: steps K of this image */
    int32_t status;           /* filled: this image's status */
} ibip_job;

/* The whole path for n images of any sizes in one call: EDT, invasion
 * (Section 2.1), trapping (Section 2.2.3) when `trapped` is given, and the
 * saturation / Pc curve (Sections 2.2.1-2.2.2; computed from seq_out when
 * trapping ran, else from seq) when `sat_per_step` is given.  The
 * invasions of all images run in one launch, one persistent CTA per image,
 * largest first; results equal the per-image calls bit for bit.
 *   h_jobs: host array of n jobs (1 <= n <= 4096); n_steps and status are
 *           written back.  An image's pore count must stay below 2^25,
 *           the whole batch's below 2^31.
 * Synchronous.  Returns IBIP_OK when every job succeeded, else the first
 * failing job's status (IBIP_ERR_ARG with n_steps = K when K exceeded
 * capacity_steps). */
IBIP_API int ibip_invade_batched(ibip_ctx *ctx, int32_t n, ibip_job *h_jobs);

/* One image of a batched paper-literal invasion; device pointers unless
 * stated, the caller owns every buffer.  Outputs as ibip_invade_literal. */
typedef struct {
    const uint8_t *image;     /* uint8[N] pore image */
    ibip_dims dims;
    int32_t inlet;            /* ibip_face */
    const int32_t *dt2;       /* int32[N] squared EDT, or NULL (computed) */
    int64_t max_steps;        /* < 0: no limit */
    int32_t *seq;             /* int32[N] output */
    int32_t *cstep;           /* int32[N] output */
    int32_t *step_r2;         /* int32[capacity_steps] output */
    int32_t *step_count;      /* int32[capacity_steps] output */
    int64_t capacity_steps;
    int64_t n_steps;          /* filled: steps K */
    int32_t status;           /* filled: this image's status */
} ibip_literal_job;

/* The paper-literal invasion (ibip_invade_literal, Section 2.1 as printed)
 * for n images of any sizes: the set-up of every image, then one launch in
 * which each image runs on a thread-block cluster of its own (CTA 0 of the
 * cluster keeps the image's bucket bookkeeping, every CTA stamps a share of
 * each step's spheres), then the final pass of every image.  The CTAs per
 * cluster come from ibip_set_literal_cluster, else, with autotuning on
 * (ibip_set_autotune), from timing 1, 2, 4, 8 and 16 on the first call of
 * each batch shape (image count, total voxels to a power of two), else
 * enough to fill the SMs.  Results equal ibip_invade_literal per image bit
 * for bit.  1 <= n <= 4096.  *h_cluster (if not NULL) gets the cluster size
 * run (the fastest one when this call tuned; fewer CTAs than asked when the
 * device cannot place the cluster with the batch's bucket bookkeeping; 0
 * when some image's bookkeeping exceeds shared memory and the images ran
 * one at a time).  Synchronous; returns IBIP_OK when every image
 * succeeded, else the first failing image's status. */
IBIP_API int ibip_invade_literal_batched(ibip_ctx *ctx, int32_t n, ibip_literal_job *h_jobs, int *h_cluster);

/* CTAs per image cluster of ibip_invade_literal_batched: 1, 2, 4, 8 or 16,
 * or 0 for the automatic choice. */
IBIP_API int ibip_set_literal_cluster(ibip_ctx *ctx, int cluster);

/* ---- serving: a continuous-batching request loop ----------------------
 * A server owns one device arena of mem_budget bytes and max_slots worker
 * slots, each a host thread with its own non-blocking stream.  Submitted
 * jobs wait in arrival order; the job at the head is admitted as soon as a
 * slot is idle and a contiguous piece of the arena large enough for its
 * scratch (ibip_job_footprint) is free.  An admitted job runs the same path
 * as ibip_invade_batched does for one image (EDT, invasion, trapping when
 * `trapped` is given, the curve when `sat_per_step` is given), on its
 * slot's stream, so the jobs in flight overlap on the device; its results
 * equal those of the one-image calls bit for bit.  Its scratch stays
 * resident in the arena until it completes, then the piece is returned. */
typedef struct ibip_server ibip_server;

typedef struct {
    int32_t status;          /* the job's ibip_status */
    int32_t slot;            /* slot that ran it */
    int64_t n_steps;         /* steps K */
    int64_t t_submit_ns;     /* host steady-clock times: submitted, */
    int64_t t_start_ns;      /*   admitted, */
    int64_t t_end_ns;        /*   results complete on the device */
    int64_t mem_reserved;    /* arena bytes held while it ran */
    int64_t mem_used;        /* arena bytes its scratch actually took */
} ibip_result;

/* Upper bound of the scratch bytes one job of these dimensions takes
 * (including a dt2 buffer when the job gives none). */
IBIP_API int64_t ibip_job_footprint(ibip_dims dims, int with_dt2);

/* Creates a server on ctx's device (ctx itself is not used afterwards).
 * 1 <= max_slots <= 128.  Allocates the arena (IBIP_ERR_OOM if it cannot).
 * Each slot has two streams: its wide kernels (EDT, rank sort, curve) at
 * the device's lowest stream priority, its one-CTA invasion and the
 * per-round widest-path launches at the highest; its waits sleep on
 * blocking-sync events.  CUDA maps streams onto CUDA_DEVICE_MAX_CONNECTIONS
 * hardware queues (8 by default): with more streams than queues a long
 * invasion kernel holds up the later launches of every stream sharing its
 * queue, so set CUDA_DEVICE_MAX_CONNECTIONS=32 in the environment before
 * the process creates its CUDA context and keep 2 * max_slots <= 32 (the
 * Python binding sets it when imported first).  Measured on the 600-request
 * stream (20 req/s, 64^3-384^3): 13.5 images/s served with 8 queues, 20.9
 * with 32. */
IBIP_API int ibip_server_create(ibip_server **out, ibip_ctx *ctx, size_t mem_budget, int max_slots);

/* Waits for every submitted job, stops the slots and frees the arena. */
IBIP_API int ibip_server_destroy(ibip_server *srv);

/* Queues a job (validated as in ibip_invade_batched; a job whose footprint
 * exceeds the whole arena is IBIP_ERR_OOM) and returns its ticket.  The
 * job's buffers must stay valid until it completes.  Thread-safe. */
IBIP_API int ibip_server_submit(ibip_server *srv, const ibip_job *job, uint64_t *h_ticket);

/* *h_done = 1 and *h_result filled when the job has completed, else 0.
 * A completed ticket can be polled again until the server is destroyed.
 * Thread-safe. */
IBIP_API int ibip_server_poll(ibip_server *srv, uint64_t ticket, int *h_done, ibip_result *h_result);

/* As ibip_server_poll, waiting up to timeout_us microseconds (< 0: no
 * limit) for the job to complete. */
IBIP_API int ibip_server_wait(ibip_server *srv, uint64_t ticket, int64_t timeout_us, int *h_done,
                              ibip_result *h_result);

/* Counters: [submitted, completed, running, waiting, arena bytes in use,
 * arena bytes, peak jobs running at once, peak arena bytes in use, kernel
 * launches queued by the slots]; n <= 9. */
IBIP_API int ibip_server_stats(ibip_server *srv, int64_t *h_stats, int n);

/* ---- serving replicas on several GPUs ----------------------------------
 * The invasion of one image is a serial chain of steps (Section 2.1: each
 * step's sphere depends on the previous stamp), so several GPUs serve a
 * request stream by taking whole requests.  A router holds one server
 * (above) per replica -- a device, which may be listed more than once --
 * and sends each request to the replica with the least outstanding work:
 * the voxels of the jobs submitted to it and not yet seen complete, among
 * the replicas whose arena can hold the job (ibip_job_footprint); ties go
 * to the lowest replica index.  No collective and no peer memory: a job
 * runs on its replica's device alone. */
typedef struct ibip_router ibip_router;

/* The routing rule by itself (host only, no device): the index i with the
 * smallest h_load[i] among those with h_capacity[i] >= footprint, the
 * lowest such index on ties; IBIP_ERR_OOM when none can hold it,
 * IBIP_ERR_ARG for n < 1, NULL arrays or footprint < 0. */
IBIP_API int ibip_route_pick(int n, const int64_t *h_load, const int64_t *h_capacity, int64_t footprint);

/* One server of mem_budget bytes and max_slots slots per entry of
 * h_devices[n] (1 <= n <= 64), each with a context of its own.  Errors as
 * ibip_server_create. */
IBIP_API int ibip_router_create(ibip_router **out, int n, const int *h_devices, size_t mem_budget,
                                int max_slots);

/* Waits for every submitted job and frees every replica. */
IBIP_API int ibip_router_destroy(ibip_router *router);

/* The replica (and its device, if h_device is not NULL) that a job of these
 * dimensions should go to now (with_dt2: the job gives no dt2 buffer, as
 * for ibip_job_footprint).  Place the job's buffers on that device, then
 * call ibip_router_submit.  Thread-safe. */
IBIP_API int ibip_router_route(ibip_router *router, ibip_dims dims, int with_dt2, int *h_replica,
                               int *h_device);

/* Queues a job on replica `replica` (as ibip_server_submit; its buffers
 * must be on that replica's device) and returns a router ticket. */
IBIP_API int ibip_router_submit(ibip_router *router, int replica, const ibip_job *job, uint64_t *h_ticket);

/* As ibip_server_wait for a router ticket; *h_replica (if not NULL) gets the
 * replica that ran it. */
IBIP_API int ibip_router_wait(ibip_router *router, uint64_t ticket, int64_t timeout_us, int *h_done,
                              ibip_result *h_result, int *h_replica);

/* Counters of one replica: [device, jobs routed to it, outstanding voxels,
 * then the 9 counters of ibip_server_stats]; n <= 12. */
IBIP_API int ibip_router_stats(ibip_router *router, int replica, int64_t *h_stats, int n);

/* Wait for everything queued on the context's stream; returns the first
 * error seen. */
IBIP_API int ibip_synchronize(ibip_ctx *ctx);

/* Number of libibip kernel launches queued on this context so far. */
IBIP_API int64_t ibip_launch_count(const ibip_ctx *ctx);

/* Kernel classes timed by the profiler. */
typedef enum {
    IBIP_K_EDT = 0,       /* the three EDT passes of ibip_edt / ibip_invade */
    IBIP_K_RANK = 1,      /* rank sort and bit-plane setup of ibip_invade */
    IBIP_K_INVADE = 2,    /* the persistent invasion kernel */
    IBIP_K_MAXIMIN = 3,   /* widest-path propagation rounds (trapping, opening) */
    IBIP_K_TRAP = 4,      /* trapped mask, seq_out and re-ranking */
    IBIP_K_PC = 5,        /* histogram, scan, saturation and Pc */
    IBIP_K_DILATE = 6,    /* per-level dilation passes of the opening */
    IBIP_K_NCLASSES = 7
} ibip_kernel_class;

/* Turn per-kernel timing on (nonzero) or off.  Turning it on clears the
 * log.  While on, each kernel class is bracketed by a pair of CUDA events on
 * the context's stream (events recorded: at most 65536 pairs). */
IBIP_API int ibip_profile_enable(ibip_ctx *ctx, int on);

/* Synchronise the stream and report, for kernel class `cls`, the summed
 * device time in milliseconds (*h_ms) and the number of bracketed spans
 * (*h_spans) since profiling was enabled. */
IBIP_API int ibip_profile_read(ibip_ctx *ctx, int cls, double *h_ms, int64_t *h_spans);

/* Counters of the context's last ibip_invade / ibip_invade_ex call, for
 * tracing (cycles are SM clock cycles counted by thread 0 of the invasion
 * CTA).  The cycle entries are measured only by calls made while a trace is
 * set (ibip_invade_trace), which run a separate, timed build of the loop;
 * otherwise they read 0 (the clock reads would cost the loop about a tenth
 * of its time).  Writes up to n (at most 48) of:
 *   0 steps, 1 status, 2 iterations of the main loop,
 *   3-5 cycles selecting, bounding (candidate shell) and committing,
 *   6 batch items taken, 7 batch items committed, 8 stale summary bits
 *   cleared, 9 ball rows committed,
 *   10-11 cycles and count of main-loop batches of single-voxel balls,
 *   12-15 select sub-phase cycles (gather, item data, pairwise tests,
 *   bookkeeping), 16-18 select / bound / commit cycles of those batches,
 *   19-21 iterations, steps and cycles of the single-voxel loop,
 *   22-23 bookkeeping sub-phases (containment rounds, row prefix),
 *   24-25 bound stages 1 (shell listing) and 2 (rank lookups),
 *   26-27 commit stage 1 (stamping) and the rest (queueing),
 *   28-29 and 33 the single-voxel loop's gather, bound and commit cycles,
 *   30-32 rounds (0 on the work queue, none counted in per-round
 *   launches), tile activations and relaxation
 *   sweeps of the context's last widest-path propagation (trapping or the
 *   opening's trim),
 *   34 out-of-range accesses counted by a checked build (IBIP_CHECKED),
 *   35 rank of the first voxel with the smallest dt2,
 *   36 batches seen by the trace (ibip_invade_trace; counted beyond its
 *   capacity), 37 the kernel's span in SM cycles, 38 the same span in
 *   nanoseconds of the global timer (their ratio is the SM clock),
 *   39-41 shell rows, listed shell candidates and removed candidates,
 *   summed over the main loop's batches, 42 batches of one item committed
 *   by the single-pass path, 43-44 batches of the single-voxel loop formed
 *   by merging (no bitmap gather) and their selection cycles, 45-46
 *   rounds of the bitmap gathers and gathers. */
IBIP_API int ibip_invade_stats(const ibip_ctx *ctx, int64_t *h_stats, int n);

/* Per-batch timing trace of later ibip_invade / ibip_invade_ex calls on
 * this context (diagnostics; the paper has no counterpart: it measures the
 * per-step cost of the sequential invasion of Section 2.1 on this design).
 * d_trace: device array of capacity_records records of eight int32 each,
 * 16-byte aligned, owned by the caller and kept alive while tracing is on:
 * {first step of the batch (0-based), steps it committed, SM cycles from
 * its selection to the end of its commit, loop (0 main, 1 single-voxel),
 * items taken, ball rows stamped (steps in the single-voxel loop), shell
 * rows scanned, shell candidates listed (both 0 in the single-voxel loop)}.
 * Records past the capacity are counted (stats entry 36), not written.
 * d_trace == null turns tracing off.  Returns IBIP_ERR_ARG for a negative
 * capacity or a misaligned array.  Batched calls are never traced. */
IBIP_API int ibip_invade_trace(ibip_ctx *ctx, int32_t *d_trace, int64_t capacity_records);

/* Tile-shape autotuning (a tuning aid around the method; the paper has no
 * counterpart).  mode 1: the first squared EDT of each shape class (every
 * dimension rounded up to a power of two, and the GPU's SM count) times
 * every candidate tile shape on that call's own input -- the candidates
 * compute the same dt2, so the call's result does not change -- and keeps
 * the fastest for later calls of that class; mode 0 (the default) uses the
 * built-in shape.  Results are shared by all contexts of the process.
 * cache_path (may be null): a text file of earlier results, read now and
 * appended to with each new result, one line "<key> <choice> <us>".
 * Returns IBIP_ERR_ARG for another mode or a path of 512 bytes or more. */
IBIP_API int ibip_set_autotune(ibip_ctx *ctx, int mode, const char *cache_path);

/* Force the EDT tile shape of this context: z_warps rows per block in the
 * z pass and strip_warps warps per block in the y and x passes, one of the
 * candidates (8,16) (4,16) (16,16) (8,8) (4,8) (16,8); (0,0) returns to the
 * tuned or built-in shape.  IBIP_ERR_ARG for any other pair. */
IBIP_API int ibip_set_edt_tiles(ibip_ctx *ctx, int z_warps, int strip_warps);

/* The tile shape an EDT of these dimensions uses on this context now
 * (forced, tuned, or the built-in (8,16)). */
IBIP_API int ibip_edt_tiles(ibip_ctx *ctx, ibip_dims dims, int *h_z_warps, int *h_strip_warps);

/* Cancel (on = 1) the invasion running on this context, or the next one
 * it starts; on = 0 withdraws the request.  Safe to call from another host
 * thread while ibip_invade / ibip_invade_ex / ibip_invade_batched block.
 * The flag lives in host-mapped memory; the invasion kernel reads it every
 * 16 batches of its main loop and every 64 of its single-voxel loop, and
 * stops before committing the next batch: the call returns
 * IBIP_ERR_CANCELLED with *h_n_steps = k, and seq, step_r2 and step_centre
 * hold a valid invasion of k steps, which ibip_invade_ex(resume = 1)
 * continues to the same result as an uninterrupted call.  Serving the
 * request clears the flag; the context stays usable.  An invasion that
 * ends before it reads the flag returns normally and leaves the flag set
 * (withdraw it with on = 0).  The paper has no counterpart (a control path
 * around the method). */
IBIP_API int ibip_cancel(ibip_ctx *ctx, int on);

/* Test hook (fault injection on the host): the nth scratch allocation of
 * this context from now that needs new device memory fails, so the call
 * that makes it returns IBIP_ERR_OOM (its outputs are then undefined, as
 * after any error); later calls allocate again and the context stays
 * usable.  nth = 0 turns the hook off; a negative nth is IBIP_ERR_ARG.
 * The paper has no counterpart. */
IBIP_API int ibip_debug_fail_alloc(ibip_ctx *ctx, int nth);

/* Static text for a status code. */
IBIP_API const char *ibip_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* IBIP_H */

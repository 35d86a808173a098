/*
 * dco_stereo.h -- C ABI of the GB300 (sm_103a) AD-census stereo matcher.
 *
 * The matcher is the sparse-depth stage of the depth contour occlusion
 * method of arXiv 2203.02300 ("Mixed Reality Depth Contour Occlusion Using
 * Binocular Similarity Matching and Three-dimensional Contour
 * Optimisation"), Sect. 4: a rectified RGB pair goes in, a sparse disparity
 * map comes out.  Steps: census transform and AD measure (Sect. 4.2.1),
 * cross-support arms (Sect. 4.1), the robust exponential AD+census cost with
 * the adaptive weight alpha (Eq. 1), aggregation over the adaptive filter
 * area (Eq. 2), winner-take-all (Eq. 3) and outlier removal by a left-right
 * consistency check (Sect. 4.3, Sect. 7.4).
 *
 * Conventions shared by every entry point
 *   - Images are interleaved RGB uint8, row-major, pitch 3*W bytes, no
 *     padding (pixel (x, y) channel c at byte 3*(y*W + x) + c).
 *   - Disparities are int16, row-major W*H, d in [d_min, d_min + D - 1]
 *     (p->d_min, 0 by default); -1 = invalid (rejected by the consistency
 *     check).
 *   - Kernels are launched with programmatic stream serialization (each
 *     waits for the preceding work of its stream before touching memory),
 *     so a launch overlaps the end of the previous one on the stream.
 *   - "device" pointers must be CUDA device memory (or managed memory) of
 *     the device the handle was created on; "host" pointers are ordinary
 *     (preferably pinned) host memory.  The caller owns every buffer it
 *     passes; the library never frees or retains them after the call.
 *   - Work is enqueued on `stream` (a cudaStream_t passed as void*; NULL =
 *     the legacy default stream) and returns before it completes, except
 *     where stated.  Output buffers are valid once the stream reaches the
 *     call's completion.
 *   - A handle owns one workspace.  Calls on one handle must not run
 *     concurrently (use one handle per stream that works in parallel).
 *   - Argument errors return DCO_EINVAL before anything is enqueued.
 *     Limits: 1 <= W, H <= 16384; 1 <= D; 0 <= p->d_min; d_min + D <= 256
 *     and <= W (D counts the disparities searched, d_min + D - 1 is the
 *     largest; maps hold absolute disparities); 1 <= arm_l1 <= 40;
 *     census window odd, at most 64 bits; lambda_ad, lambda_census, eps > 0;
 *     gamma_l >= 0.
 *   - A workspace the device cannot allocate returns DCO_ENOMEM (one beyond
 *     the handle's budget DCO_EBUDGET) before anything is enqueued; the
 *     handle stays usable, and its next calls allocate what they need.
 *   - Device-side failures do not trap: they set the handle's status word,
 *     read with dco_stereo_sync_status() or dco_stereo_stream_status().  The
 *     vertical pass sets bit 0 when a TMA tile copy does not complete within
 *     its bounded mbarrier wait (reported as DCO_ETIMEOUT; the block stops
 *     issuing copies and returns), and so does the cost pass when its
 *     staging bulk copies do not; bit 1 when the vertical pass's shared
 *     memory is not 128-byte aligned for the copies (DCO_EDEVICE); the
 *     pass's outputs are then not valid.
 */
#ifndef DCO_STEREO_H
#define DCO_STEREO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dco_stereo dco_stereo; /* opaque handle: device, workspace, tables */
typedef void *dco_stream;             /* cudaStream_t */

typedef enum {
    DCO_OK = 0,
    DCO_EINVAL = 1,   /* bad argument (size, pointer, parameter) */
    DCO_ENOMEM = 2,   /* device allocation failed */
    DCO_EBUDGET = 3,  /* the call needs more workspace than the handle's budget */
    DCO_ECUDA = 4,    /* a CUDA runtime call failed */
    DCO_ETIMEOUT = 5, /* a bounded device-side wait gave up */
    DCO_EDEVICE = 6   /* a kernel reported an internal bound-check failure */
} dco_status;

/*
 * Matcher parameters.  lambda_ad, lambda_census, gamma_l, eps are the
 * paper's (Eq. 1; values of Sect. 7.2: 10, 40, 1, 0.8).  The census window,
 * the arm rule constants and the consistency tolerance are not given in the
 * paper; the defaults are this library's reading:
 *   census 9x7 on the grey level Y = (77R + 150G + 29B + 128) >> 8, centre
 *   excluded, clamp-to-edge, bit k = [Y(neighbour) < Y(p)] in window
 *   row-major order;
 *   arms (Sect. 4.1, colour + distance double threshold): the arm in one
 *   direction is the largest k <= arm_l1 such that every step j <= k stays in
 *   the image, has max-channel difference < tau1 to p and to step j-1, and,
 *   when j > arm_l2, < tau2 to p (defaults 34, 17, 20, 6);
 *   lr_tol = 1 (a negative value disables the consistency check);
 *   vote_iters = 0: rounds of the parallax optimisation of Sect. 4.3 (Eq. 4)
 *   applied to the checked map (see dco_stereo_vote), 0..64;
 *   smooth_arms = 0: with 1, the "morphological processing" of Sect. 4.1 is
 *   read as a grey-level opening (3x3 minimum, then 3x3 maximum, windows cut
 *   to the image) of each arm map; L_min, alpha and the support regions then
 *   follow the opened arms (dco_stereo_arms returns them too);
 *   agg_order = 0: the order of the two 1-D sums of the cross-region
 *   aggregation (Sect. 4.2.2, Eq. 2).  0: horizontal sums along each pixel's
 *   horizontal arm, then their sum over p's vertical arm (region = union
 *   over q on p's vertical arm of q's horizontal segment).  1: vertical sums
 *   first, then their sum over p's horizontal arm (region = union over q on
 *   p's horizontal arm of q's vertical segment).  In both, N(p) of Eq. 2 is
 *   the size of the region actually summed.  The Eq. 4 vote always counts
 *   over the order-0 region.
 */
typedef struct {
    float lambda_ad;
    float lambda_census;
    float gamma_l;
    float eps;
    int census_w;
    int census_h;
    int arm_l1;
    int arm_l2;
    int tau1;
    int tau2;
    int lr_tol;
    int d_chunk; /* disparities aggregated per pass (0 = automatic); see dco_stereo_match */
    int vote_iters; /* Eq. 4 rounds after the consistency check (0 = none) */
    int smooth_arms; /* 1: smooth cross-support window (Sect. 4.1), see above; 0 = raw arms */
    int agg_order; /* 0: horizontal then vertical sums (Eq. 2); 1: vertical then horizontal */
    int d_min; /* smallest disparity searched (Eq. 3's d_min): d in [d_min, d_min + D - 1]; 0 */
    int h_chunk; /* tile: scan positions per block of the first 1-D pass (0 = automatic); see below */
    int v_chunk; /* tile: output positions per block of the second 1-D pass (0 = automatic) */
} dco_params;

/* Fill *p with the defaults above.  DCO_EINVAL if p is NULL. */
dco_status dco_params_default(dco_params *p);

/* Human-readable name of a status code (static string, never NULL). */
const char *dco_status_string(dco_status s);

/*
 * Create a handle on CUDA device `device`.  `workspace_budget_bytes` caps
 * the device memory the handle may allocate for its workspace (0 = no
 * cap).  The workspace grows on demand (a synchronising reallocation) or is
 * sized up front by dco_stereo_reserve().  *out is NULL on failure.
 */
dco_status dco_stereo_create(dco_stereo **out, int device, size_t workspace_budget_bytes);

/* Release the handle and its workspace.  NULL is accepted.  Synchronises
 * the device before freeing. */
void dco_stereo_destroy(dco_stereo *h);

/*
 * Device bytes of workspace one match of a W x H pair with D disparities
 * needs under params p (0 if the arguments are invalid).  Per pixel: two
 * 16-byte census/colour records, two arm words, the running best cost and
 * disparity of both views; per pixel and per disparity of one pass: the
 * two horizontal-aggregate slices (4 bytes each).  Never the full
 * W x H x D cost volume.
 */
size_t dco_stereo_workspace_bytes(int W, int H, int D, const dco_params *p);

/* Allocate the workspace for (W, H, D, p) now.  DCO_EBUDGET if it exceeds
 * the handle's budget. */
dco_status dco_stereo_reserve(dco_stereo *h, int W, int H, int D, const dco_params *p);

/*
 * The whole hot path for one rectified pair (Sect. 4.1-4.3):
 *   census + grey + arms for both views -> Eq. 1 costs -> Eq. 2 horizontal
 *   then vertical aggregation over the cross-support region -> Eq. 3 WTA
 *   for the left- and right-reference views -> left-right check ->
 *   p->vote_iters rounds of the Eq. 4 parallax optimisation (left view).
 * left, right: device, W*H*3 bytes.  disp_out: device, W*H int16.
 * The disparity range is processed in passes of p->d_chunk disparities
 * (automatic when 0) so the workspace holds slices, never the volume.
 * Tile shapes (they change the speed, never the result): the first 1-D
 * pass (rows for agg_order 0, columns for 1) splits each line into blocks
 * of p->h_chunk outputs (0: whole lines up to 1024 positions, else 512;
 * otherwise 32 <= h_chunk, capped at 1024 - 2 arm_l1 below the line); the second
 * pass splits each line into balanced blocks of at most p->v_chunk outputs
 * (0: whole lines up to 512 positions, else blocks of at most 432; otherwise
 * 32 <= v_chunk, capped at 512 - 2 arm_l1).  Each block reads arm_l1
 * positions of halo on both sides.
 * p = NULL uses the defaults.
 */
dco_status dco_stereo_match(dco_stereo *h, const uint8_t *left, const uint8_t *right,
                            int W, int H, int D, const dco_params *p,
                            int16_t *disp_out, dco_stream stream);

/*
 * As dco_stereo_match, with the per-view results.  Any output may be NULL.
 *   disp_left / disp_right: device W*H int16, Eq. 3 for the left / right
 *     reference view before the consistency check;
 *   cost_left / cost_right: device W*H float, the minimum aggregated cost
 *     (Eq. 2 value at the chosen disparity).
 */
dco_status dco_stereo_match_views(dco_stereo *h, const uint8_t *left, const uint8_t *right,
                                  int W, int H, int D, const dco_params *p,
                                  int16_t *disp_out, int16_t *disp_left, int16_t *disp_right,
                                  float *cost_left, float *cost_right, dco_stream stream);

/*
 * As dco_stereo_match, with host buffers left/right (W*H*3 bytes each) and
 * disp_host (W*H int16); waits for the stream before returning.  When all
 * three are device-accessible (pinned, registered or managed host memory,
 * reached over NVLink-C2C on Grace systems) and p->vote_iters is 0, the
 * kernels read the images and write the map in place; otherwise the images
 * are copied to the handle's device staging buffers and the map back.
 */
dco_status dco_stereo_match_host(dco_stereo *h, const uint8_t *left_host,
                                 const uint8_t *right_host, int W, int H, int D,
                                 const dco_params *p, int16_t *disp_host, dco_stream stream);

/*
 * Stage a1 alone (Sect. 4.2.1): census strings of one image.
 * rgb: device W*H*3 bytes.  census_out: device W*H uint64 (bits above
 * census_w*census_h-2 are zero).
 */
dco_status dco_stereo_census(dco_stereo *h, const uint8_t *rgb, int W, int H,
                             const dco_params *p, uint64_t *census_out, dco_stream stream);

/*
 * Stage a2 alone (Sect. 4.1): the four arm lengths of one image.
 * arms_out: device W*H*4 bytes, per pixel {left, right, up, down}.
 */
dco_status dco_stereo_arms(dco_stereo *h, const uint8_t *rgb, int W, int H,
                           const dco_params *p, uint8_t *arms_out, dco_stream stream);

/*
 * Eq. 2 aggregated costs of one reference view for every disparity
 * (diagnostic; materialises the volume).  view 0 = left reference
 * (match q = p - d), 1 = right reference (match q = p + d).
 * vol_out: device D*H*W float, index (d*H + y)*W + x.
 */
dco_status dco_stereo_cost_volume(dco_stereo *h, const uint8_t *left, const uint8_t *right,
                                  int W, int H, int D, const dco_params *p, int view,
                                  float *vol_out, dco_stream stream);

/*
 * Parallax optimisation alone (Sect. 4.3, Eq. 4), p->vote_iters rounds:
 *   d'(p) = argmax_d hist(d, N_p)
 * over the valid pixels of the support region N_p of Eq. 2 (the arms of
 * `rgb`, the reference image, under p's arm parameters); the smallest d on
 * equal counts.  Pixels of disp_in outside [p->d_min, p->d_min + D - 1]
 * (-1 = invalid) cast no vote and are written as -1.  Each round reads the whole previous map.
 * rgb: device W*H*3 bytes; disp_in, disp_out: device W*H int16 (may be the
 * same buffer).  0 rounds copies the map.  Same errors as dco_stereo_match.
 */
dco_status dco_stereo_vote(dco_stereo *h, const uint8_t *rgb, const int16_t *disp_in, int W, int H, int D,
                           const dco_params *p, int16_t *disp_out, dco_stream stream);

/*
 * Quarter-size input alone (Sect. 4): out (device (W/2)*(H/2)*3 bytes) gets
 * the rounded 2x2 channel means of rgb (device W*H*3 bytes), as used by
 * dco_stereo_depth.  W, H in [2, 32768].
 */
dco_status dco_stereo_downscale(dco_stereo *h, const uint8_t *rgb, int W, int H, uint8_t *out,
                                dco_stream stream);

/*
 * Sparse depth at full size (Sect. 4 and 4.4): the pair is reduced to half of
 * each axis (every channel the rounded mean (a + b + c + d + 2) >> 2 of its
 * 2x2 block; an odd last row or column is dropped), matched there over D
 * disparities exactly as dco_stereo_match (both views, consistency check,
 * p->vote_iters Eq. 4 rounds), and each half-size disparity d is doubled back
 * and converted with the binocular parameters: Z = f_px * baseline / (2 d)
 * written to the 2x2 block it covers; 0 marks missing depth (d <= 0, an odd
 * last row or column), the convention of Eq. 14.
 * left, right: device W*H*3 bytes (full size).  depth_out: device W*H float,
 * Z in the unit of `baseline`.  disp_half_out: optional device (W/2)*(H/2)
 * int16, the half-size map.  f_px > 0 in pixels of the full image,
 * baseline > 0.  W, H >= 2 and (W/2, H/2, D) must satisfy the limits of
 * dco_stereo_match; otherwise DCO_EINVAL.
 */
dco_status dco_stereo_depth(dco_stereo *h, const uint8_t *left, const uint8_t *right, int W, int H, int D,
                            const dco_params *p, double f_px, double baseline, float *depth_out,
                            int16_t *disp_half_out, dco_stream stream);

/*
 * Depth densification (Sect. 6, Eqs. 13-20): the dense map D minimising
 *   lambda_d  sum_p w_sparse(p) (D(p) - D_sparse(p))^2
 * + lambda_s  sum_p sum_{q in N4(p)} w_pq (D(p) - D(q))^2
 * + lambda_s2 sum_p w_stable(p) (D(p) - D_pre(p))^2
 * with w_sparse = [D_sparse > 0], w_stable = [D_pre > 0], w_pq = 0 when
 * exactly one of p, q is on the depth contour, else max(1 - min(s_p, s_q), 0),
 * s = M_fuse * M_I (Eq. 17); N4 is cut at the border.  Solved on the device
 * by Jacobi-preconditioned conjugate gradients until the residual of the
 * normal equations is below tol relative to their right-hand side, or
 * max_iters; pixels whose smoothness-connected part holds no data stay 0.
 */
typedef struct {
    float lambda_d;   /* 0.80 (Sect. 7.2) */
    float lambda_s;   /* 1.20 */
    float lambda_s2;  /* 0.02 */
    float tol;        /* 1e-5 */
    int max_iters;    /* 4000 */
    int solver;       /* 0: the whole solve in one cooperative launch when
                         every block's share of the pixels fits one block
                         (about 0.93 M pixels on 152 multiprocessors), else
                         two launches per iteration; 1: always two launches
                         per iteration.  Same iterations and stopping rule. */
} dco_dense_params;

dco_status dco_dense_params_default(dco_dense_params *p);

/*
 * d_sparse: device W*H float, 0 = no sparse depth (e.g. dco_stereo_depth's
 * output).  contour: device W*H bytes, nonzero on the depth contour B_dp, or
 * NULL (no contour).  m_fuse, m_int: device W*H float, the fused flow
 * magnitude and the [0, 1]-normalised Canny intensity of Eq. 17, or NULL (0).
 * d_pre: device W*H float, the previous frame's depth, or NULL (no stability
 * term).  d_out: device W*H float.  p = NULL uses the defaults.  The call
 * waits for the solve (with solver 1 it reads a convergence flag between
 * batches of iterations); dco_stereo_densify_stats gives the iterations run
 * and the final relative residual.  Needs 36 bytes per pixel of workspace.
 * DCO_ETIMEOUT if a grid barrier of the one-launch solve gave up (its waits
 * are bounded); the map is then not a solution.  The call cannot be
 * captured in a CUDA graph (DCO_EINVAL under capture).
 */
dco_status dco_stereo_densify(dco_stereo *h, const float *d_sparse, const uint8_t *contour, const float *m_fuse,
                              const float *m_int, const float *d_pre, int W, int H, const dco_dense_params *p,
                              float *d_out, dco_stream stream);

dco_status dco_stereo_densify_stats(dco_stereo *h, int *iters, double *rel_residual);

/*
 * Stage a7 alone: left-right consistency.  out(x,y) = dl(x,y) if
 * x - dl >= 0 and |dl - dr(x - dl, y)| <= tol, else -1; tol < 0 copies dl.
 * dl, dr, out: device W*H int16.  The handle is only used for its device.
 */
dco_status dco_stereo_lr_check(dco_stereo *h, const int16_t *dl, const int16_t *dr,
                               int W, int H, int tol, int16_t *out, dco_stream stream);

/* One pair of a batch (all pointers device).  d_chunk: this pair's pass
 * width (disparities aggregated per pass, e.g. chosen per shape by an
 * autotuner); 0 takes p->d_chunk of the call.  Under a workspace budget the
 * library may narrow it further, as for a single pair. */
typedef struct {
    const uint8_t *left;
    const uint8_t *right;
    int W, H, D;
    int16_t *disp_out;
    int d_chunk;
    int h_chunk, v_chunk; /* this pair's tile shapes (0: the call's p->h_chunk / v_chunk) */
} dco_pair_desc;

/*
 * Match n independent pairs of possibly different W, H, D in one pass of
 * the pipeline: each stage is one launch over all pairs.  The workspace
 * holds all pairs' per-pixel buffers and one pass of slices for each.
 * Results equal dco_stereo_match on each pair alone (bit-identical).
 * descs: host array of n descriptors.
 * Admission under the handle's budget: when the pairs' workspaces do not fit
 * the budget together even at the narrowest pass width (32 disparities),
 * the pairs are admitted in consecutive groups that do fit, run one group
 * after the other on `stream` in the same workspace (the allocation never
 * exceeds the budget; dco_stereo_batch_groups gives the group count).  A
 * single pair that does not fit returns DCO_EBUDGET before anything is
 * enqueued.
 */
dco_status dco_stereo_match_batch(dco_stereo *h, const dco_pair_desc *descs, int n,
                                  const dco_params *p, dco_stream stream);

/* Admission groups the last dco_stereo_match_batch call ran in (1 when all
 * pairs fit the budget together). */
int dco_stereo_batch_groups(dco_stereo *h);

/* Bytes of device workspace the handle currently holds (0 before its first
 * call); never above the handle's budget. */
size_t dco_stereo_workspace_allocated(dco_stereo *h);

/*
 * Waits for all work of the handle's device, then reads and clears the
 * device status word.  DCO_OK; DCO_ETIMEOUT if a copy of the cost or the
 * vertical pass did not complete within its bounded wait; DCO_EDEVICE if a kernel
 * reported another failed internal check since the last read.
 */
dco_status dco_stereo_sync_status(dco_stereo *h);

/*
 * As dco_stereo_sync_status, ordered on `stream` instead of the whole
 * device: the word is read once the work enqueued on `stream` before this
 * call has completed (the call waits for it), then cleared on `stream`.
 * Work of the handle enqueued on other streams is not waited for.
 */
dco_status dco_stereo_stream_status(dco_stereo *h, dco_stream stream);

/*
 * Failure tests (not for normal use).  DCO_TEST_LOSE_TILE_COPIES: the
 * cost pass's staging and the vertical pass's tiles arm their mbarriers but
 * issue no copy, and wait only a few polls, so every wait runs out with
 * nothing in flight; the kernels set bit 0 of the status word and return,
 * and the stream status reads DCO_ETIMEOUT.  DCO_TEST_LOSE_GRID_ARRIVAL: in the one-launch
 * densification solve, block 0 never arrives at the first grid barrier and
 * every barrier waits only a few polls, so all blocks give up and return;
 * dco_stereo_densify returns DCO_ETIMEOUT.  0 restores normal operation.
 * Unknown bits: DCO_EINVAL.
 */
#define DCO_TEST_LOSE_TILE_COPIES 1
#define DCO_TEST_LOSE_GRID_ARRIVAL 4
dco_status dco_stereo_set_test_flags(dco_stereo *h, int flags);

/*
 * The whole path of dco_stereo_match for callers that cannot allocate
 * device memory (for example code running where cudaMalloc is forbidden
 * or unavailable, or a host that must keep its memory footprint fixed after
 * start-up).  It takes no handle and allocates nothing: its workspace and
 * tables live in one 32 MiB device array built into the library, which
 * every GPU that loads the library holds until the process exits.  The
 * paper has no counterpart; this is an integration entry point.
 *   - Runs on the calling thread's current CUDA device.  The first call on a
 *     device looks up the array's device address; make that first call
 *     before any stream capture.
 *   - Sizes whose workspace (passes of 32 disparities) does not fit the
 *     array return DCO_EBUDGET before anything is enqueued: roughly
 *     W*H <= 80 000 pixels (e.g. 320x240) at any D <= 256.
 *   - All calls share the one array and it keeps the last call's contents;
 *     nothing in it needs to start at zero (every word a kernel reads was
 *     written earlier in the same call; the tables are written by a kernel
 *     that receives them by value, so no host buffer outlives the call).
 *     Calls that overlap on the GPU (other streams, other threads) race on
 *     it: serialise them.
 *   - A device-side failure (see the status word above) sets a status word
 *     in the array, which keeps its bits across calls until
 *     dco_stereo_noalloc_status reads and clears it; disp_out of a call
 *     whose status is not DCO_OK is not valid.
 * left, right: device W*H*3 bytes; disp_out: device W*H int16; p = NULL
 * uses the defaults (p->d_chunk is ignored).
 */
dco_status dco_stereo_match_noalloc(const uint8_t *left, const uint8_t *right, int W, int H, int D,
                                    const dco_params *p, int16_t *disp_out, dco_stream stream);

/*
 * Status of the allocation-free entry point on the current device: waits
 * for the work enqueued on `stream` before this call, reads the status word
 * of the static array, clears it (on `stream`) and returns DCO_OK,
 * DCO_ETIMEOUT or DCO_EDEVICE as dco_stereo_sync_status does.  Allocates
 * nothing.  Like the first dco_stereo_match_noalloc call, a first call on a
 * device looks up the array's address: make it before any stream capture.
 */
dco_status dco_stereo_noalloc_status(dco_stream stream);

/*
 * Native serving runtime: frames of several camera streams, each of its own
 * W x H x D (and pass width), submitted from host memory and matched by
 * continuous batching.  A scheduler thread admits pending frames in arrival
 * order into a batch while the frame's stream has a free device slot and the
 * batch's workspace (dco_stereo_workspace_bytes of its frames) fits a lane's
 * share of the memory budget, and runs the batch on a free lane: a handle
 * with its own workspace and CUDA stream copies the images in, runs
 * dco_stereo_match_batch (the whole path of dco_stereo_match for every
 * frame) and copies each map straight into the caller's buffer.  Frames that
 * arrive while other batches are on the device are admitted as slots and
 * lanes free up, so their work overlaps on the device.  One completion
 * thread per lane retires that lane's batches on their events and wakes the
 * callers, so a short batch is never held up behind a longer one on another
 * lane.  Streams marked latency-critical (dco_stream_desc.priority = 1, e.g.
 * the smaller frame sizes: shortest job first) are admitted first, batched
 * only with each other, and run on the lane's CUDA stream of the greatest
 * priority, so the block scheduler gives their kernels the SMs ahead of a
 * larger frame's blocks already waiting on the device.
 * Results equal dco_stereo_match on each frame alone (bit for bit).
 *
 * dco_server_create: streams[nstreams] the stream shapes (d_chunk, h_chunk,
 *   v_chunk 0: the params' pass width and tiles); lanes 1..16; slots_per_stream >= 1 (frames of one
 *   stream in flight at once); max_batch >= 1 frames per batch;
 *   budget_bytes the device workspace of all lanes together (0: every
 *   stream's frame in every lane's batch).  The server allocates its slots
 *   and warms every lane up before returning (no allocation while serving).
 *   DCO_EBUDGET if a lane's share cannot hold one frame of the largest
 *   stream.
 * dco_server_submit: left, right (W*H*3 bytes) and disp_out (W*H int16) are
 *   host buffers of the stream's shape that must stay valid until
 *   dco_server_wait returns for the ticket; returns at once with the
 *   request's ticket.  When all three are device-accessible (pinned,
 *   registered or managed memory) and p->vote_iters is 0, the kernels read
 *   and write them in place; otherwise they are copied through the
 *   stream's device slots.
 * dco_server_wait: blocks until the request is done (timeout_ms < 0: no
 *   limit; DCO_ETIMEOUT when the limit passes first, the request still
 *   pending), fills *times (may be NULL) and returns the request's status
 *   (a failed batch fails its requests; the server keeps serving).  Each
 *   ticket is waited for once.
 * dco_server_destroy: launches and retires every pending frame, then frees
 *   the server.
 * The paper has no counterpart: this is the serving pattern of the
 * matcher's deployment (several camera streams, Sect. 7's mixed-reality
 * use).
 */
typedef struct dco_server dco_server;
typedef struct {
    int W, H, D;
    int d_chunk;
    int h_chunk, v_chunk; /* tile shapes of the stream's frames (0: the params') */
    int priority;         /* 1: latency-critical stream (see above); 0: normal */
} dco_stream_desc;
typedef struct {
    double arrival_s;  /* submit time, steady clock seconds */
    double launch_s;   /* its batch was enqueued on a lane */
    double done_s;     /* the completion thread saw the batch finish */
    float device_ms;   /* the batch's copies and match on the lane's stream */
} dco_request_times;

dco_status dco_server_create(dco_server **out, int device, const dco_stream_desc *streams, int nstreams,
                             int lanes, int slots_per_stream, int max_batch, size_t budget_bytes,
                             const dco_params *p);
dco_status dco_server_submit(dco_server *s, int stream, const uint8_t *left, const uint8_t *right,
                             int16_t *disp_out, unsigned long long *ticket);
dco_status dco_server_wait(dco_server *s, unsigned long long ticket, int timeout_ms, dco_request_times *times);
/* batches launched, frames in them, the largest batch workspace and a lane's
 * budget share (any pointer may be NULL) */
dco_status dco_server_counters(dco_server *s, unsigned long long *batches, unsigned long long *frames,
                               size_t *max_batch_bytes, size_t *lane_budget);
void dco_server_destroy(dco_server *s);

/* Text of the last CUDA or budget error seen by the handle ("" if none).
 * Owned by the handle, valid until its next call. */
const char *dco_stereo_last_error(dco_stereo *h);

/*
 * Per-kernel timing.  When enabled, every kernel the handle launches is
 * bracketed by CUDA events on its stream.  After the stream has finished,
 * dco_stereo_profile_get returns, per kernel name, the number of launches
 * and their summed duration in milliseconds.
 */
dco_status dco_stereo_set_profiling(dco_stereo *h, int enable);

/* Number of kernels the handle has launched since it was created. */
unsigned long long dco_stereo_launch_count(dco_stereo *h);
dco_status dco_stereo_profile_reset(dco_stereo *h);
int dco_stereo_profile_count(dco_stereo *h);
dco_status dco_stereo_profile_get(dco_stereo *h, int i, const char **name, int *launches,
                                  double *total_ms);

#ifdef __cplusplus
}
#endif

#endif /* DCO_STEREO_H */

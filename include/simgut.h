/* simgut.h -- C-ABI of the GB300 (sm_103a) renderer for 3DGUT-style Gaussian
 * scenes into pinhole / OpenCV-fisheye cameras and spinning LiDAR, after
 * "SimULi: Real-Time LiDAR and Camera Simulation with Unscented Transforms"
 * (arXiv 2510.12901).
 *
 * Conventions for every entry point
 * ---------------------------------
 * - Status codes, never exceptions, exit() or device traps.  On failure a
 *   message is available from sg_last_error() (thread-local).
 * - Pointers named d_* are device pointers (CUDA global memory of the current
 *   device); pointers named h_* are host pointers.  All arrays are dense,
 *   row-major, float32 unless stated.
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *   stream).  Work is enqueued on it; a call returns once its work is
 *   enqueued.  The render calls read back the number of (tile, Gaussian)
 *   pairs and the device status word (below) and so wait for the depth
 *   stage of their own work; nothing else synchronises.
 * - Device status.  The sort stages wait on one another's published counts
 *   (decoupled look-back).  Every such wait is bounded; one that runs out
 *   sets the frame's status word, leaves every later kernel of the render in
 *   bounds (the tile lists come out empty) and surfaces as SG_ERR_TIMEOUT:
 *   from the render call itself when the depth sort gave up (exact mode),
 *   otherwise from sg_frame_status, sg_frame_sync_outputs, the synchronous
 *   host-output renders and the request server.
 * - Handles (scene, camera, lidar, frame) are owned by the library; create /
 *   destroy them from one host thread at a time.  Output and gradient
 *   buffers are owned by the caller.
 */
#ifndef SIMGUT_H
#define SIMGUT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SG_OK = 0,
    SG_ERR_INVALID = -1,   /* bad argument; nothing was enqueued */
    SG_ERR_OOM = -2,       /* device allocation failed */
    SG_ERR_CUDA = -3,      /* a CUDA call failed; see sg_last_error() */
    SG_ERR_OVERFLOW = -4,  /* a capacity (pairs, requests) was exceeded */
    SG_ERR_TIMEOUT = -5,   /* a bounded device wait gave up */
    SG_ERR_BUSY = -6       /* serving queue full */
} sg_status;

typedef struct sg_scene_s *sg_scene;
typedef struct sg_camera_s *sg_camera;
typedef struct sg_lidar_s *sg_lidar;
typedef struct sg_frame_s *sg_frame;

enum { SG_FEATURES_RGB = 0, SG_FEATURES_SH = 1, SG_FEATURES_LIDAR = 2, SG_FEATURES_LIDAR_SH = 3 };
enum { SG_CAMERA_PINHOLE = 0, SG_CAMERA_FISHEYE = 1 };
/* Sensor kinds of a request or a workspace query. */
enum { SG_REQ_CAMERA = 0, SG_REQ_LIDAR = 1 };

/* Library version and the CUDA architecture it was built for (103 for sm_103a). */
int sg_version(void);
int sg_cuda_arch(void);
const char *sg_last_error(void);
/* Number of CUDA kernels this library has launched in this process so far
 * (all threads); the difference across a region counts its launches. */
int64_t sg_launch_count(void);
/* Number of device and pinned-host allocation and free calls (cudaMalloc,
 * cudaFree, cudaMallocHost, cudaFreeHost) this library has made in this
 * process so far (all threads). */
int64_t sg_alloc_count(void);

/* ----------------------------------------------------------------------
 * Gaussian scene (Sec. 3.1: particles with mean mu, opacity sigma and
 * covariance Sigma = R S S^T R^T; camera particles carry degree-<=3 SH colour,
 * LiDAR particles carry features zeta = (intensity, beta_hit, beta_drop)).
 * ---------------------------------------------------------------------- */
typedef struct {
    int64_t n;                 /* number of Gaussians, >= 0 */
    const float *d_means;      /* [n,3] world metres */
    const float *d_log_scales; /* [n,3] log of the per-axis standard deviation */
    const float *d_quats;      /* [n,4] (w,x,y,z); normalised by the library */
    const float *d_opacity;    /* [n] in (0,1), already activated */
    const float *d_features;   /* [n,F]: RGB F=3, SH F=3*(deg+1)^2 laid out
                                  [n,(deg+1)^2,3], LiDAR F=3, LiDAR SH
                                  F=3*(deg+1)^2 laid out as SH */
    int feature_kind;          /* SG_FEATURES_* */
    int sh_degree;             /* 0..3, used with SG_FEATURES_SH and _LIDAR_SH */
} sg_gaussians_desc;
/* Feature kinds.  SH (camera colour): c = max(sum_k Y_k(d) c_k + 0.5, 0),
 * evaluated once per Gaussian at the direction d from the camera centre to
 * the mean.  LIDAR: zeta = the three floats as given.  LIDAR_SH (the SH^l
 * of Sec. 3.1): zeta = sum_k Y_k(d) c_k with neither offset nor clamp (an
 * intensity and two logits), evaluated once per Gaussian at the direction
 * from the sensor origin of the column pose that sees the mean to the mean.
 * Y_k: real spherical harmonics of degree <= 3, orthonormal on the sphere. */

/* Copies the caller's arrays (device pointers, caller keeps ownership) into a
 * library-owned planar layout on `stream`.  The caller's arrays may be freed
 * once the stream has passed this call.  Errors: SG_ERR_INVALID (n<0, NULL
 * array with n>0, bad kind/degree), SG_ERR_OOM, SG_ERR_CUDA. */
sg_status sg_create_scene(const sg_gaussians_desc *desc, void *stream, sg_scene *out);
/* Overwrites the parameters of an existing scene with the same n and feature
 * layout (a training step).  Same errors as sg_create_scene. */
sg_status sg_update_scene(sg_scene scene, const sg_gaussians_desc *desc, void *stream);
/* sg_destroy_*: wait for the device's queued work, then free (a render
 * still queued may read the object).  A frame keeps referring to the scene
 * and sensor of its last render: destroy it, or render again, before them
 * if it is to be used again. */
void sg_destroy_scene(sg_scene scene);
int64_t sg_scene_size(sg_scene scene);

/* Dynamic actors (Sec. 3.1, scene graph).  Gaussian i belongs to actor
 * d_actor_of[i] (0..n_actors-1) or to the static background (-1).  An
 * actor's Gaussians have their means and quaternions (as given to
 * sg_create_scene / sg_update_scene) in the actor's frame; every render
 * first maps them to the world with the actor's current pose (its SE(3) at
 * the render's timestamp): mu_w = Ra mu + t, R_w = Ra R.  Their SH (colour
 * or SH^l) are evaluated at the view direction expressed in the actor's
 * frame, so the appearance turns with the object.  The backward returns the
 * gradients in each Gaussian's own frame.
 *
 * sg_scene_set_actors: d_actor_of [n] int32 (device, copied; ignored when
 *   n_actors = 0, which makes every Gaussian static again).  Every pose
 *   starts as the identity.  The call waits for `stream` (renders still
 *   queued on it may read the old lists) and checks the indices.  Errors:
 *   SG_ERR_INVALID (NULL scene, n_actors < 0, NULL list, an index outside
 *   -1..n_actors-1), SG_ERR_OOM, SG_ERR_CUDA, SG_ERR_BUSY (during a capture).
 * sg_scene_set_actor_poses: h_poses [n_actors,12] row-major [R | t], actor
 *   to world (host memory, R a rotation).  The copy is queued on `stream`:
 *   renders queued on `stream` after the call use the new poses.  Renders
 *   on other streams must be ordered after it by the caller, and no render
 *   may still be reading the previous poses when it runs.  Errors:
 *   SG_ERR_INVALID (NULL argument, a scene without actors, a non-finite
 *   entry), SG_ERR_CUDA. */
sg_status sg_scene_set_actors(sg_scene scene, const int32_t *d_actor_of, int n_actors,
                              void *stream);
sg_status sg_scene_set_actor_poses(sg_scene scene, const float *h_poses, void *stream);

/* ----------------------------------------------------------------------
 * Camera (Sec. 3.2: arbitrary camera models through the unscented
 * transform).  Pixel (i,j) is the ray through (i+0.5, j+0.5); OpenCV axes
 * (x right, y down, z forward).  Fisheye: theta_d = theta (1 + k1 t^2 + k2 t^4
 * + k3 t^6 + k4 t^8), valid incidence angles [0, theta_max] with theta_max the
 * first stationary point of theta_d (at most pi/2); pixels beyond it carry no
 * ray.  Builds a per-pixel ray table in double precision on the device
 * (synchronous).  Errors: SG_ERR_INVALID (size <= 0 or > 16384, f <= 0, bad
 * model), SG_ERR_OOM, SG_ERR_CUDA.
 * ---------------------------------------------------------------------- */
sg_status sg_create_camera(int model, int width, int height, float fx, float fy,
                           float cx, float cy, const float k[4], sg_camera *out);
void sg_destroy_camera(sg_camera cam);

/* ----------------------------------------------------------------------
 * Spinning LiDAR (Sec. 3.3; App. A Proc. 1 ElevationTiling; App. B ray-based
 * culling).  Beams have elevations h_elev_deg[n_beams] (degrees); column c
 * has azimuth az0_deg + (c+0.5)*360/n_cols in the sensor frame (x forward,
 * y left, z up).  The elevation tiling (n_elev_tiles = N_phi, at most
 * max_rays_per_tile = M rays per tile), the azimuth tile count N_theta, the
 * ray-to-tile assignment and the summed-area table of the ray mask over a
 * dense grid of cull_az x (n_elev_tiles * cull_el_per_tile) cells are
 * computed once here and reused by every render (synchronous).
 * Errors: SG_ERR_INVALID (n_beams or n_cols <= 0 or > 65535, N_phi out of
 * [1,1024], M <= 0, cull sizes <= 0, more than 65535 tiles), SG_ERR_OOM.
 * ---------------------------------------------------------------------- */
sg_status sg_create_lidar(const float *h_elev_deg, int n_beams, int n_cols, float az0_deg,
                          int max_rays_per_tile, int n_elev_tiles, int cull_az,
                          int cull_el_per_tile, sg_lidar *out);
void sg_destroy_lidar(sg_lidar lidar);
/* Tiling results: h_T receives n_elev_tiles+1 elevation boundaries (degrees);
 * *n_theta the azimuth tile count.  Either pointer may be NULL. */
sg_status sg_lidar_tiling(sg_lidar lidar, float *h_T, int *n_theta);

/* ----------------------------------------------------------------------
 * Render options.  Defaults (sg_default_opts): alpha_min 1/255, alpha_max
 * 0.99, t_min 1e-4, near 0.2 m, unscented transform (alpha,beta,kappa) =
 * (1,2,0), 2 LiDAR pose iterations, ray-based culling on.
 * ---------------------------------------------------------------------- */
typedef struct {
    float alpha_min, alpha_max, t_min, near_dist;
    float ut_alpha, ut_beta, ut_kappa;
    int pose_iters;   /* LiDAR: fixed-point iterations choosing each sigma
                         point's column pose (0..8) */
    int cull;         /* LiDAR: ray-based culling (App. B) on/off */
    float beam_divergence; /* LiDAR: beam divergence delta in radians, 0 (default) = off,
                              at most 0.1.  Eq. 6: a LiDAR Gaussian's covariance becomes
                              Sigma + (delta r)^2 (I - d d^T), r and d the distance and
                              direction from the origin of the column pose that sees its
                              mean; the opacity is not rescaled.  The UT takes its sigma
                              points along the Cholesky columns of that covariance. */
} sg_render_opts;
sg_render_opts sg_default_opts(void);

/* ----------------------------------------------------------------------
 * Frame: the workspace of one render and the state the backward pass needs
 * (per-Gaussian projection, sorted (tile, Gaussian) lists, per-ray final
 * transmittance and contributor counts).  Buffers grow on demand.  A frame
 * serves one render at a time; sg_backward_* reads the last render.
 * ---------------------------------------------------------------------- */
sg_status sg_frame_create(sg_frame *out);
void sg_frame_destroy(sg_frame frame);
/* Whether renders with this frame write the per-ray state the backward
 * reads (final transmittance, sums, contributor count: 36 bytes per ray);
 * on (1) by default.  A frame used for forward renders only (inference,
 * serving) can turn it off (0) and save that memory traffic;
 * sg_backward_* then refuses the frame's renders (SG_ERR_INVALID), and
 * the SG_FIELD_RAY_STATE / SG_FIELD_N_CONTRIB fields are not updated.
 * Camera renders of such a frame use a compositing kernel that tracks no
 * backward state and parameterises each ray in its tile's tangent plane
 * (fewer operations per ray-Gaussian pair): its images equal the
 * state-keeping kernel's up to float rounding, not bit for bit, and are
 * deterministic from one render to the next.
 * Errors: SG_ERR_INVALID (NULL frame). */
sg_status sg_frame_set_backward_state(sg_frame frame, int keep);

/* Capacity mode.  With max_pairs > 0 the frame's (tile, Gaussian) pair
 * buffers are sized for max_pairs pairs and sg_render_camera /
 * sg_render_lidar no longer wait for the pair count: nothing in the call
 * synchronises with the device (after the first call at a given size has
 * allocated the workspace), so a render can be captured into a CUDA graph.
 * Pairs beyond max_pairs are dropped, which leaves the result incomplete:
 * after the render has completed, sg_frame_dropped_pairs tells.  Because
 * the pose travels through pinned memory owned by the frame, a render in
 * capacity mode must have completed before the next render call on the
 * same frame.  max_pairs = 0 restores the default (exact) mode.  Errors:
 * SG_ERR_INVALID (NULL frame, max_pairs < 0 or >= 2^31). */
sg_status sg_frame_set_capacity(sg_frame frame, int64_t max_pairs);
/* After a capacity-mode render on `frame` has completed: the pairs kept
 * (*pairs, may be NULL) and the pairs dropped for want of room (*dropped;
 * 0 = the result is complete).  SG_ERR_INVALID in exact mode. */
sg_status sg_frame_dropped_pairs(sg_frame frame, int64_t *dropped, int64_t *pairs);

/* Device status of the frame's last render: copies the status word on
 * `stream` (the stream of that render, or one ordered after it) and waits
 * for it.  SG_OK, or SG_ERR_TIMEOUT when a bounded look-back wait of the
 * sort stages ran out in that render (its tile lists were left empty, so
 * its outputs show no Gaussian).  SG_ERR_INVALID for a frame never
 * rendered or a frame of sg_render_camera_static. */
sg_status sg_frame_status(sg_frame frame, void *stream);

/* ----------------------------------------------------------------------
 * Workspace query for admission (a serving loop's memory budget).  The
 * device bytes a frame's buffers grow to for one render of `scene` into a
 * sensor of kind sensor_kind (SG_REQ_CAMERA or SG_REQ_LIDAR) with n_rays
 * rays: the per-Gaussian projection and sort buffers and per-ray state,
 * which are exact, and the (tile, Gaussian) pairs with their sort scratch,
 * masks and compositing work items for an allowance of
 * SG_ADMIT_PAIRS_PER_GAUSSIAN pairs per Gaussian (a render that makes more
 * pairs grows past the estimate), with the library's growth head-room.  The
 * tile count is bounded from n_rays: 16x16-pixel camera tiles of images at
 * least 256 pixels on a side, LiDAR tiles of at least SG_ADMIT_LIDAR_RAYS_PER_TILE
 * rays.  Errors: SG_ERR_INVALID (NULL scene or bytes, unknown kind, n_rays < 0).
 * sg_frame_workspace_bytes: the bytes a frame holds now (device buffers).
 * ---------------------------------------------------------------------- */
#define SG_ADMIT_PAIRS_PER_GAUSSIAN 4
#define SG_ADMIT_LIDAR_RAYS_PER_TILE 8
sg_status sg_workspace_bytes(sg_scene scene, int sensor_kind, int64_t n_rays, size_t *bytes);
sg_status sg_frame_workspace_bytes(sg_frame frame, size_t *bytes);

/* ----------------------------------------------------------------------
 * Testing hook for the device status path (not needed in normal use).
 * max_spins: polling rounds a look-back wait makes before it gives up
 * (0 = the default, about a second).  hold_site / hold_tile: the kernel
 * kind and the tile (ticket) whose published counts are withheld, so that
 * the next tile's wait is certain to run out (hold_site 0: none).  Every
 * wait stays bounded and every access in bounds.  The values live in the
 * current device's memory (so that replays of captured CUDA graphs see
 * them); the call synchronises that device first.  Set them back with
 * (0, SG_LOOKBACK_NONE, -1) after use. */
enum {
    SG_LOOKBACK_NONE = 0,
    SG_LOOKBACK_COMPACT = 1,     /* depth stage: compaction of the visible Gaussians */
    SG_LOOKBACK_DEPTH_SORT = 2,  /* depth stage: radix passes over the depth keys */
    SG_LOOKBACK_OFFSETS = 3,     /* depth stage: scan of the tile counts into pair offsets */
    SG_LOOKBACK_TILE_SORT = 4    /* radix passes over the pairs' tile ids */
};
sg_status sg_debug_lookback(uint32_t max_spins, int hold_site, int64_t hold_tile);
/* Testing hook for the device status path (not needed in normal use):
 * give_up != 0 makes the camera projection's first wait for its bulk copies
 * of SH planes give up at once (status word set, SG_ERR_TIMEOUT from the
 * render); a second bounded wait still precedes every read of the staged
 * planes, so the render stays in bounds.  0 restores the normal wait.  The
 * value lives in the current device's memory; the call synchronises that
 * device first.  Errors: SG_ERR_CUDA. */
sg_status sg_debug_bulk_wait(int give_up);

/* ----------------------------------------------------------------------
 * Forward render (Eq. 1: front-to-back compositing of alpha_i = sigma_i
 * rho_i(tau_max) over the per-tile list sorted by (tile, depth, id); Sec. 3.2
 * projection of 7 sigma points; Sec. 3.3 LiDAR).
 *
 * Camera: h_c2w[12] is the row-major 3x4 camera-to-world pose [R | t] (host
 * memory, read during the call).  Outputs (device, may be NULL):
 *   d_rgb [H,W,3]  premultiplied foreground colour sum_i c_i alpha_i T_i
 *   d_alpha [H,W]  omega = sum_i alpha_i T_i
 *   d_depth [H,W]  sum_i tau_i alpha_i T_i / omega, 0 where omega = 0
 * LiDAR: d_col_c2w [n_cols,12] per-column sensor-to-world poses (device,
 * 16-byte aligned).
 * Outputs (device, may be NULL), [n_beams, n_cols] beam-major:
 *   d_range    sum_i tau_i alpha_i T_i / omega (0 where omega = 0)
 *   d_intensity first channel of zeta
 *   d_drop      softmax(beta_hit, beta_drop) probability of a drop
 *   d_alpha     omega
 * Errors: SG_ERR_INVALID (NULL handle / pose, misaligned poses, opts out of range, LiDAR
 * features on a camera render or vice versa), SG_ERR_OOM, SG_ERR_CUDA,
 * SG_ERR_OVERFLOW (more than 2^31-1 pairs), SG_ERR_TIMEOUT (a look-back wait
 * of the depth sort gave up; later ones are reported by sg_frame_status).
 * ---------------------------------------------------------------------- */
sg_status sg_render_camera(sg_scene scene, sg_camera cam, const float h_c2w[12],
                           const sg_render_opts *opts, sg_frame frame, float *d_rgb,
                           float *d_alpha, float *d_depth, void *stream);
sg_status sg_render_lidar(sg_scene scene, sg_lidar lidar, const float *d_col_c2w,
                          const sg_render_opts *opts, sg_frame frame, float *d_range,
                          float *d_intensity, float *d_drop, float *d_alpha,
                          void *stream);

/* Rolling-shutter camera render (Sec. 3.2, time-dependent effects: sensor
 * motion in the projection and each ray evaluated with its own time).
 * d_row_c2w [H,12] (device, the caller keeps it valid until the render and
 * any sg_backward_camera of this frame have run): the row-major [R | t]
 * camera-to-world pose of every pixel row at its exposure time.  A pixel's
 * ray takes its row's origin and rotation; a point's pixel is computed with
 * the pose of the row it falls in, found from the middle row by taking the
 * pose of the row the point projects to, opts->pose_iters times (clamped to
 * the image); the depth key and the SH direction use the row that sees the
 * mean.  Outputs and errors as sg_render_camera (SG_ERR_INVALID for NULL row
 * poses, or a frame of sg_render_camera_static). */
sg_status sg_render_camera_rs(sg_scene scene, sg_camera cam, const float *d_row_c2w,
                              const sg_render_opts *opts, sg_frame frame, float *d_rgb,
                              float *d_alpha, float *d_depth, void *stream);

/* Same renders with host output buffers: the device result is copied to
 * h_* (pinned or pageable) on `stream` and the call waits for it (and
 * returns SG_ERR_TIMEOUT if a look-back wait of the render gave up).  Inputs
 * stay as above except the LiDAR poses, which are read from host memory. */
sg_status sg_render_camera_host(sg_scene scene, sg_camera cam, const float h_c2w[12],
                                const sg_render_opts *opts, sg_frame frame, float *h_rgb,
                                float *h_alpha, float *h_depth, void *stream);
sg_status sg_render_lidar_host(sg_scene scene, sg_lidar lidar, const float *h_col_c2w,
                               const sg_render_opts *opts, sg_frame frame, float *h_range,
                               float *h_intensity, float *h_drop, float *h_alpha,
                               void *stream);

/* ----------------------------------------------------------------------
 * Several camera views of one scene in one call: a vehicle's camera rig
 * rendered per frame (the paper's evaluation renders the three front
 * cameras of every frame, Sec. 4).  Each view is the render sg_render_camera
 * makes of it, with identical results, on the view's own stream and frame.
 * The call first starts every view (projection, depth sort, pair count),
 * then finishes them in order (binning, tile sort, compositing), so that
 * while the host waits for one view's pair count the other views' kernels
 * are already queued: views on different streams overlap on the GPU.
 *
 * views[i]: camera; row-major 3x4 camera-to-world pose (copied); frame
 * (distinct for every view); output buffers rgb [H,W,3], alpha [H,W],
 * depth [H,W] (each may be NULL); stream; row_c2w (NULL, or the per-row
 * poses of a rolling-shutter view).  host_outputs = 0: the outputs
 * are device buffers and the call returns with the work queued, as
 * sg_render_camera.  host_outputs = 1: the outputs are host buffers
 * (pinned or pageable); each view's result is copied there on its stream
 * and the call returns once every view's copy is done.  host_outputs = 2:
 * as 1, but the call returns with the copies queued (pinned buffers copy
 * asynchronously); the caller calls sg_frame_sync_outputs on a view's frame
 * before it reads or reuses that view's host buffers.  The copies run on a
 * stream of the frame's own, after the view's render, so that the view's
 * stream goes on to its next work; the frame's next render waits for them.
 * SG_ERR_INVALID for another value.  Errors as for
 * sg_render_camera, and SG_ERR_INVALID for n_views < 0, a NULL list,
 * camera or frame, or two views sharing a frame; after an error, views
 * already started may still run on their streams. */
typedef struct {
    sg_camera camera;
    float c2w[12];
    sg_frame frame;
    float *rgb, *alpha, *depth;
    void *stream;
    const float *row_c2w;   /* device [H,12]: a rolling-shutter view as
                               sg_render_camera_rs (c2w unused); NULL: global */
} sg_camera_view;
sg_status sg_render_cameras(sg_scene scene, int n_views, const sg_camera_view *views,
                            const sg_render_opts *opts, int host_outputs);
/* Wait until the host copies of the frame's last render with host outputs
 * are done (at once if it has none).  SG_ERR_TIMEOUT if a look-back wait of
 * that render gave up (the copies are done all the same). */
sg_status sg_frame_sync_outputs(sg_frame frame);

/* ----------------------------------------------------------------------
 * Camera render that allocates nothing.  The paper has no counterpart: this
 * is a deployment variant of sg_render_camera for callers that must not
 * allocate device memory while they run (for example when another
 * allocator already holds the device's memory, or when the implicit
 * device-wide synchronisation of cudaMalloc / cudaFree is not acceptable in
 * their loop).  The whole workspace lives in one file-scope device array of
 * about 17 MB that every GPU which loads the library keeps until the process
 * exits.  Limits: at most 32768 Gaussians, 65536 pixels (256 tiles of
 * 16x16) and 262144 (tile, Gaussian) pairs; larger inputs return
 * SG_ERR_INVALID (sizes) or SG_ERR_OVERFLOW (pairs) with a message.
 * Arguments and outputs are those of sg_render_camera without the frame:
 * no state is kept for a backward pass.  The first call on a device looks
 * up the array's device address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.  All calls
 * share the one array: calls that overlap on the GPU (other threads or
 * streams of the same device) race and must be serialised by the caller.
 * Nothing in the array needs clearing between calls: every stage writes the
 * parts it later reads.  Like sg_render_camera, the call waits once for the
 * pair count; SG_ERR_TIMEOUT when a look-back wait of the depth sort gave
 * up.  (A wait of the tile sort that gives up leaves the lists empty and is
 * not reported: the call keeps no frame to query.)  The call makes no
 * allocation of any kind: sg_alloc_count does not change across it.
 * ---------------------------------------------------------------------- */
sg_status sg_render_camera_static(sg_scene scene, sg_camera cam, const float h_c2w[12],
                                  const sg_render_opts *opts, float *d_rgb, float *d_alpha,
                                  float *d_depth, void *stream);

/* ----------------------------------------------------------------------
 * Backward (the differentiable renderer of Sec. 3.2 / 3.4).  Given the
 * upstream gradients of the last render in `frame` (device, same shapes as
 * the outputs; NULL = zero), accumulates dL/d parameters into caller-owned
 * device arrays (NULL = not wanted): d_g_means [n,3], d_g_log_scales [n,3],
 * d_g_quats [n,4], d_g_opacity [n], d_g_features [n,F].  The caller zeroes
 * them; the call adds (float atomics, so the summation order and the last
 * bits vary run to run).  The unscented transform only selects tiles and is
 * not differentiated.  The sensor the frame was rendered with (and, for
 * LiDAR and rolling-shutter renders, the device poses) must still exist:
 * the frame refers to them.  With dynamic actors the gradients are in each
 * Gaussian's own frame.  Errors: SG_ERR_INVALID (frame not rendered from
 * this scene / sensor kind), SG_ERR_CUDA.
 * ---------------------------------------------------------------------- */
typedef struct {
    float *d_g_means, *d_g_log_scales, *d_g_quats, *d_g_opacity, *d_g_features;
} sg_grads;
sg_status sg_backward_camera(sg_scene scene, sg_frame frame, const float *d_g_rgb,
                             const float *d_g_alpha, const float *d_g_depth,
                             const sg_grads *grads, void *stream);
sg_status sg_backward_lidar(sg_scene scene, sg_frame frame, const float *d_g_range,
                            const float *d_g_intensity, const float *d_g_drop,
                            const float *d_g_alpha, const sg_grads *grads, void *stream);

/* ----------------------------------------------------------------------
 * Request server (continuous batching).  Scenes and sensors are created as
 * above and stay resident; requests reference them.  n_slots worker threads
 * each own a CUDA stream and a render workspace; a request is admitted, in
 * arrival order, when a slot is free and its estimated workspace fits in
 * memory_budget bytes next to the requests already running (0 = no
 * limit), so requests that arrive while others run start as soon as a slot
 * and memory free up, and their GPU work overlaps on separate streams.
 * Latency runs from sg_server_submit to the completion of the request's
 * last kernel.  A request's buffers (outputs, LiDAR poses) belong to the
 * caller and must stay valid until sg_server_wait returns for it.  The
 * first request of each size grows a slot's workspace (which synchronises
 * the device once); warm every slot up before measuring.  Every wait is a
 * host wait with a timeout: SG_ERR_TIMEOUT, never a hang.
 *
 * CUDA graphs (use_graphs = 1): for each (scene, sensor, options)
 * combination a slot renders its first request exactly, the second in
 * capacity mode (sg_frame_set_capacity: room for 1.25x the largest pair
 * count seen plus 64K) while capturing that launch sequence into a CUDA
 * graph, and every later one by replaying the graph: one launch and no host
 * synchronisation per request.  The pose and the output and pose pointers
 * of each request reach the graph through a small descriptor in pinned
 * memory that the graph copies to the device first.  A replay whose pairs
 * exceed the capacity is rendered again exactly (the result is always
 * complete) and the graph is captured anew with a larger capacity.
 *
 * Batching (max_batch > 1): when a request is admitted, the requests already
 * waiting (among the next 32 in the queue) of the same combination (scene,
 * sensor, options) join it, up to max_batch, as far as the memory budget
 * allows; the others keep their order.  A batch renders as one launch
 * sequence: its requests on the slot's frames, forked onto per-request
 * streams (cameras through one sg_render_cameras call), and, with graphs,
 * as one captured graph per (combination, batch size), replayed with one
 * launch.  Every request of a batch completes when the batch does.
 * ---------------------------------------------------------------------- */
typedef struct sg_server_s *sg_server;
typedef struct {
    int n_slots;            /* requests running at once, 1..64 */
    size_t memory_budget;   /* device bytes for running requests' workspaces, 0 = unlimited */
    int queue_capacity;     /* waiting requests before submit returns SG_ERR_BUSY */
    int use_graphs;         /* 1 (default): replay captured CUDA graphs, see below */
    int fifo_priority;      /* 1 (default): a request admitted behind k others in flight
                               runs on a stream of the k-th CUDA priority level (older
                               requests first); 0: all at one priority */
    int max_batch;          /* 1..16 (default 4): queued requests of the admitted one's
                               combination join it, up to this many, see below */
} sg_server_config;
typedef struct {
    int kind;                   /* SG_REQ_CAMERA or SG_REQ_LIDAR */
    sg_scene scene;
    sg_camera camera;           /* SG_REQ_CAMERA */
    sg_lidar lidar;             /* SG_REQ_LIDAR */
    float c2w[12];              /* SG_REQ_CAMERA: camera-to-world pose */
    const float *d_col_c2w;     /* SG_REQ_LIDAR: per-column poses (device) */
    float *d_out[4];            /* camera: rgb, alpha, depth; LiDAR: range,
                                   intensity, drop, alpha (device, may be NULL) */
    sg_render_opts opts;
} sg_request;
typedef struct {
    int64_t completed, failed, rays, peak_in_flight, queued;
    int64_t graph_replays;      /* requests served by replaying a captured graph */
    int64_t graph_captures;     /* graphs captured (one per slot and combination) */
    int64_t overflow_rerenders; /* replays whose pairs outgrew the capacity, redone exactly */
    int64_t batches;            /* renders that served several requests at once */
    int64_t batched_requests;   /* requests served by those */
    double latency_mean_ms, latency_p50_ms, latency_p99_ms, latency_max_ms;
    double span_s;              /* first arrival to last completion */
    double mrays_per_s;         /* rays of completed requests / span */
} sg_server_report;
sg_server_config sg_default_server_config(void);
sg_status sg_server_create(const sg_server_config *cfg, sg_server *out);
/* Enqueue a request (never blocks).  SG_ERR_BUSY when the queue is full,
 * SG_ERR_INVALID for an incomplete request or one larger than the budget. */
sg_status sg_server_submit(sg_server server, const sg_request *req, uint64_t *ticket);
/* Wait (at most timeout_s seconds, <= 0: no limit) for one request; returns
 * its render status and latency, or SG_ERR_TIMEOUT. */
sg_status sg_server_wait(sg_server server, uint64_t ticket, double timeout_s,
                         double *latency_ms);
/* Wait for every submitted request to finish (or SG_ERR_TIMEOUT). */
sg_status sg_server_drain(sg_server server, double timeout_s);
sg_status sg_server_stats(sg_server server, sg_server_report *out);
sg_status sg_server_reset_stats(sg_server server);
/* Stops the workers (requests not yet started are dropped) and frees. */
void sg_server_destroy(sg_server server);

/* ----------------------------------------------------------------------
 * Inspection of the last render's intermediate buffers, for tests and
 * profiling.  Returns a device pointer into the frame (valid until the next
 * render with it) and the element count.  Fields:
 *   SG_FIELD_RECT      float4 per Gaussian: per-ray test box x_lo,x_hi,y_lo,y_hi
 *   SG_FIELD_TILES     int4 per Gaussian: tile range x0,x1,y0,y1 (LiDAR x may wrap)
 *   SG_FIELD_DEPTH     float per Gaussian: sort key |mu - o|
 *   SG_FIELD_COUNT     uint32 per Gaussian: number of tiles binned into (0 = culled)
 *   SG_FIELD_PAIR_IDS  uint32 per pair: Gaussian id, sorted by (tile, depth, id)
 *   SG_FIELD_PAIR_TILES uint32 per pair: tile id of the same order
 *   SG_FIELD_RANGES    uint2 per tile: [start, end) into the pair list
 *   SG_FIELD_RAY_STATE float4 per ray: final transmittance, omega,
 *                      Z = sum tau_i alpha_i T_i, LiDAR drop probability
 *   SG_FIELD_N_CONTRIB uint32 per ray: list entries up to the last composited one
 *   SG_FIELD_MEAN2D    float2 per Gaussian: UT mean
 *   SG_FIELD_COV2D     float4 per Gaussian: UT covariance xx, xy, yy, 0
 * ---------------------------------------------------------------------- */
enum {
    SG_FIELD_RECT = 0, SG_FIELD_TILES = 1, SG_FIELD_DEPTH = 2, SG_FIELD_COUNT = 3,
    SG_FIELD_PAIR_IDS = 4, SG_FIELD_PAIR_TILES = 5, SG_FIELD_RANGES = 6,
    SG_FIELD_RAY_STATE = 7, SG_FIELD_N_CONTRIB = 8, SG_FIELD_MEAN2D = 9,
    SG_FIELD_COV2D = 10
};
sg_status sg_frame_field(sg_frame frame, int field, const void **d_ptr, int64_t *count);
/* Number of (tile, Gaussian) pairs (in capacity mode: those kept), tiles and
 * rays of the last render. */
sg_status sg_frame_stats(sg_frame frame, int64_t *n_pairs, int64_t *n_tiles,
                         int64_t *n_rays);

/* ----------------------------------------------------------------------
 * Per-stage timing of the last render (CUDA events on its stream), in ms:
 * [0] project, [1] depth sort + offsets, [2] bin + tile sort + ranges,
 * [3] render.  Enabled with sg_frame_set_timing(frame, 1).
 * ---------------------------------------------------------------------- */
sg_status sg_frame_set_timing(sg_frame frame, int on);
sg_status sg_frame_timing(sg_frame frame, float ms[4]);
/* The five stage boundaries of the last render of `frame` (start, after
 * projection, after the depth stage, after binning, end), in ms after the
 * start of the last render of `ref` (which may be `frame`; both timed, on
 * the same device).  Renders on several streams can so be placed on one
 * time line.  Waits for both renders. */
sg_status sg_frame_marks(sg_frame frame, sg_frame ref, float ms[5]);

#ifdef __cplusplus
}
#endif
#endif /* SIMGUT_H */

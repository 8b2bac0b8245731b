/*
 * rr.h -- C ABI of the GB300 radar scan simulator (RadaRays method,
 * Mock, Magnusson, Hertzberg, arXiv 2310.03505).
 *
 * The library simulates a rotating FMCW radar by ray tracing, as Sec. III of
 * the paper describes: for every azimuth beam it samples rays from the D3
 * cone (Sec. III-A, Eq. 2), traces them through a triangle scene over several
 * bounces with a Fresnel split into reflected and refracted rays (Sec. III-A),
 * collects the energy that returns to the sensor through the beam window of
 * the material lobe (Eq. 3-5), sums the returns by range into a polar image
 * (Sec. III-B) and applies the blur / beam-pattern / noise pass (Sec. III-C).
 *
 * Conventions shared by every entry point
 *  - Status: every function returns RR_OK (0) or one of the RR_ERR_* codes
 *    below; no C++ exception crosses this boundary.  rr_last_error() gives a
 *    message for the last failure on the calling thread.  On failure nothing
 *    is written to the output buffers.
 *  - Pointers: "host or device" arguments may point to host memory (pageable
 *    or pinned) or to CUDA device memory of the current device; the library
 *    tells them apart with cudaPointerGetAttributes.  The caller owns every
 *    buffer it passes; the library copies what it needs.
 *  - Streams: work is issued on the stream set with rr_set_stream() from the
 *    calling thread (default: the legacy default stream).  Blocking calls
 *    synchronise that stream before they return.
 *  - Layout of the polar image: float32, row major [n_azimuth][n_bins]
 *    (azimuth major), linear energy; each azimuth emits E0 = 1 (Sec. III-A:
 *    the ray energies of a beam sum to the emitted energy).
 *  - Threads: a scene may be used from several threads, but calls on the same
 *    scene are serialised by the caller (the scene owns its scan workspace).
 */
#ifndef RR_H
#define RR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RR_VERSION 1

/* status codes */
#define RR_OK 0
#define RR_ERR_INVALID_ARG 1 /* a size, index, pointer or parameter is out of range     */
#define RR_ERR_OOM 2         /* a device allocation failed                              */
#define RR_ERR_CAPACITY 3    /* the ray tree outgrew the scan workspace (see message)   */
#define RR_ERR_TIMEOUT 4     /* a bounded device wait gave up                           */
#define RR_ERR_CUDA 5        /* a CUDA runtime call failed                              */
#define RR_ERR_BUSY 6        /* the request cannot be admitted now                      */
#define RR_ERR_CANCELLED 7   /* the request was cancelled before it ran                 */

/* sensor flags (rr_sensor_params.flags) */
#define RR_MULTIPATH 1u  /* air-path returns, Sec. III-A ("multi-path reflection")   */
#define RR_REFRACTION 2u /* trace the refracted child, Sec. III-A                     */
#define RR_SPECKLE 4u    /* multiply each return by an Exp(1) draw                    */
#define RR_NOISE 8u      /* uniform system and ambient noise, Sec. III-C              */
#define RR_COUNT_TRAVERSAL 16u /* count BVH nodes visited and triangles tested (stats) */
#define RR_NOISE_PERLIN 32u    /* with RR_NOISE: Perlin instead of uniform noise, Sec. III-C */

/* material flags (rr_material.flags) */
#define RR_MAT_PERFECT_CONDUCTOR 1u /* R = 1, T = 0 whatever the angle            */
/* Lobe of the beam window (Eq. 4) other than Eq. 5 (Sec. III-A: user-defined
   BRDFs per material).  The lobe is a symmetric density over the deviation w
   from the mirror direction on [-pi/2, pi/2], normalised to unit integral. */
#define RR_MAT_COOK_TORRANCE 2u  /* the microfacet lobe of the paper's Sec. IV: A = diffuse
                                    amount kd, B = Beckmann roughness m > 0; f(w) = kd cos(w)/2
                                    + (1 - kd) D(w/2) / Zw, D the Beckmann distribution of the
                                    half-vector angle w/2, Zw its integral (closed form) */
#define RR_MAT_TABULATED_LOBE 4u /* the density set by rr_scene_set_lobe (until then Eq. 5 with
                                    A, B, C) */
#define RR_LOBE_SAMPLES 4097u    /* samples of a tabulated lobe: density at j (pi/2) / 4096 */

#define RR_NO_HIT 0xFFFFFFFFu

/* limits checked by the library */
#define RR_MAX_BOUNCES 16u
#define RR_MAX_BINS 16384u
#define RR_MAX_AZIMUTH 65535u
#define RR_MAX_RAYS_PER_BEAM 65535u
#define RR_MAX_MATERIALS 65535u

typedef struct rr_scene rr_scene; /* opaque: resident triangles, LBVH, lobe tables, workspace */

/* Per-material radar properties.  eps_r >= 1 is the relative permittivity
   (refractive index sqrt(eps_r), Snell and Fresnel of Sec. III-A),
   loss_tangent >= 0 sets the attenuation inside the material.  A, B, C are
   the lobe parameters of Eq. 5 with S = 1 - A - B; 0 <= A, B, A + B <= 1,
   C >= 0. */
typedef struct {
  float eps_r;
  float loss_tangent;
  float A, B, C;
  uint32_t flags;
} rr_material;

/* Sensor pose: position p (metres) and orientation q = (w, x, y, z), sensor to
   world.  q need not be exactly unit; it is normalised. */
typedef struct {
  float p[3];
  float q[4];
} rr_pose;

/* Sensor model (Sec. III-A/B/C and the setup of Sec. IV).
   n_azimuth      azimuth beams over 360 deg, beam a points at 2 pi a / n_azimuth
   rays_per_beam  N_s initial rays per beam, each with energy 1 / N_s
   max_bounces    maximum number of intersections along a path (>= 1)
   n_bins         range bins; bin i covers [i, i + 1) * bin_size_m
   beam_width_rad b of Eq. 2 and Eq. 4; beam_prob P of Eq. 2 (0 < P < 1)
   elevation_rad  elevation of the beam axes
   t_min_m        self-intersection offset: hits need t > t_min_m
   min_energy     rays carrying less energy are not spawned (0: keep all)
   freq_hz        carrier frequency (wavelength of the loss model)
   blur_sigma_bins    Gaussian blur along range (measurement noise), 0: off
   az_pattern_sigma   Gaussian beam pattern across azimuths (in beams), 0: off
   noise_sys, noise_amb amplitudes of the uniform system / ambient noise
   flags          RR_MULTIPATH | RR_REFRACTION | RR_SPECKLE | RR_NOISE | RR_NOISE_PERLIN
   seed, scan_id  key and counter words of the Philox4x32-10 draws
   beam_aspect    elliptic beams (Sec. III-A: the cone stretched along an
                  axis): the inclination offsets of the D3 cone are scaled by
                  this factor and the receive weight of the air path follows
                  the same elliptic Gaussian; 0 or 1: circular
   noise_cell_az, noise_cell_bins  Perlin lattice spacing in azimuth beams and
                  range bins (0: 8 and 32); the lattice wraps around the circle
                  with round(n_azimuth / noise_cell_az) cells
   range_falloff  exponent k of an optional range weight of the returns: a
                  return at range r > 1 m adds its energy times (1 m / r)^k to
                  the image (Eq. 1's R^-4 power falloff with k = 4, made
                  explicit; returns nearer than 1 m are not scaled).  0 (the
                  default): the image follows the ray density alone, as
                  Sec. III-A describes.  In [0, 16]. */
typedef struct {
  uint32_t n_azimuth, rays_per_beam, max_bounces, n_bins;
  float beam_width_rad, beam_prob, elevation_rad, bin_size_m, t_min_m, min_energy, freq_hz;
  float blur_sigma_bins, az_pattern_sigma, noise_sys, noise_amb;
  uint32_t flags;
  uint64_t seed;
  uint32_t scan_id;
  float beam_aspect;
  float noise_cell_az, noise_cell_bins;
  float range_falloff;
} rr_sensor_params;

/* One traced segment (debug dump): initial ray (az, k), branch path (bit i =
   0 reflected / 1 refracted at intersection i), bounce index, original
   triangle id hit (RR_NO_HIT on a miss or beyond the range limit), hit
   distance (+inf on a miss), the energy entering the segment, and at the hit
   cos theta0 (incidence, >= 0), the energies of the traveled-path and
   air-path returns (0 on a miss), and the number of BVH nodes the query
   visited. */
typedef struct {
  uint32_t az, k, path, bounce;
  uint32_t tri;
  float t;
  float E;
  uint32_t flags; /* bit 0: an air-path visibility test ran (a candidate whose window W toward the
                     sensor and receive weight g are both non-zero in float32: otherwise its return
                     is 0 whatever the visibility), bit 1: the sensor was visible */
  float cos_i, ret_t, ret_a;
  float visits; /* BVH nodes the closest-hit query visited (diagnostics) */
} rr_segment;

typedef struct {
  uint32_t n_triangles, n_materials, bvh_depth;
  uint32_t n_wide_nodes;    /* nodes of the 8-wide quantised BVH (0 until it is first used) */
  uint64_t device_bytes;    /* scene buffers (not the scan workspace) */
  uint64_t workspace_bytes; /* current scan workspace */
  float build_ms;           /* device time of the last LBVH build */
  float reserved_f;
} rr_scene_info;

typedef struct {
  uint64_t closest_queries; /* closest-hit queries over all bounces and scans */
  uint64_t anyhit_queries;  /* air-path visibility queries */
  uint64_t returns;         /* return records written */
  uint64_t scans;
  uint64_t nodes_visited;   /* BVH nodes the closest-hit queries fetched (RR_COUNT_TRAVERSAL scans only) */
  uint64_t tris_tested;     /* triangles the closest-hit queries tested (RR_COUNT_TRAVERSAL scans only) */
  uint64_t kernel_launches; /* kernels this scene launched (host count) */
  uint64_t anyhit_nodes_visited; /* the same for the visibility queries */
  uint64_t anyhit_tris_tested;
} rr_stats;

/* kernel kinds reported by rr_profile_read */
#define RR_K_RAYGEN 0
#define RR_K_TRACE 1 /* closest-hit queries */
#define RR_K_SHADE 2 /* shading and compaction; with deferred visibility also the air-path candidates */
#define RR_K_IMAGE 3
#define RR_K_BUILD 4 /* LBVH build and the 8-wide collapse */
#define RR_K_VIS 5   /* air-path visibility queries (and, with a min_energy cut, the candidate pass) */
#define RR_K_COUNT 6
typedef struct {
  double ms[RR_K_COUNT];        /* sum of the launches' event durations */
  uint64_t launches[RR_K_COUNT];
  double busy_ms[RR_K_COUNT];   /* length of the union of the launches' event intervals: the time during
                                   which at least one launch of the kind ran.  Launches on several streams
                                   (split scans) overlap, so ms can exceed busy_ms. */
} rr_profile;

/* ---------------------------------------------------------------------- */
/* general                                                                 */
/* ---------------------------------------------------------------------- */
int rr_version(void);

/* Message of the last failed call on this thread ("" if none).  The string
   stays valid until the next call on this thread. */
const char* rr_last_error(void);

/* Stream for subsequent calls from this thread (a cudaStream_t; NULL = the
   legacy default stream). */
int rr_set_stream(void* cuda_stream);

/* Failure detection without a GPU fault.  Every spin-wait in this library's
   kernels is bounded: when the flag it waits for is not set within about a
   second, the kernel raises an error bit, stops waiting and returns, the
   call that launched it reports RR_ERR_TIMEOUT (or a failed build), and the
   CUDA context stays usable.  This call proves it for one wait: it runs the
   real kernel (or device function) of that wait, on one block, over
   counters arranged so that the awaited flag is never set, on its own
   scratch memory (no scene involved):
     RR_WAIT_TOP_TASK     a block task of the SAH-top build (k_top_sah) waits
                          for a task number that is never published while one
                          task stays pending;
     RR_WAIT_WIDE_NODE    the wide-BVH collapse (k_wide_alloc) waits for a
                          wide node that is allocated but never published;
     RR_WAIT_SHADE_PREFIX the decoupled look-back of the shading pass waits
                          for a preceding tile that never publishes.
   Returns RR_ERR_TIMEOUT when the wait gave up and raised its error bit (the
   expected outcome), RR_ERR_CUDA if the wait ended otherwise or a CUDA call
   failed, RR_ERR_INVALID_ARG for an unknown `which`.  *waited_ms (may be
   NULL) receives the wall time of the call.  Blocking; runs on the stream of
   rr_set_stream. */
#define RR_WAIT_TOP_TASK 0u
#define RR_WAIT_WIDE_NODE 1u
#define RR_WAIT_SHADE_PREFIX 2u
int rr_selftest_wait(uint32_t which, double* waited_ms);

/* Failure detection, host-side fault injection (no counterpart in the paper:
   the library's own failure handling).  Every device and pinned host
   allocation the library makes passes one gate.  fail_at >= 0 arms it: the
   allocations go on until fail_at more have passed, and the next one fails
   as if the device were out of memory (no CUDA call is made for it), after
   which the gate is disarmed again; fail_at < 0 disarms it.  The call that
   met the failure returns RR_ERR_OOM with a message naming what it was
   allocating, frees what it had allocated and leaves the library usable.
   *allocs_seen (may be NULL) receives the number of allocations that passed
   the gate since the previous call, so a test can count how many an
   operation makes.  Process-wide (all threads and devices); for tests. */
int rr_fault_inject_alloc(int64_t fail_at, uint64_t* allocs_seen);

/* ---------------------------------------------------------------------- */
/* scene: ingest + LBVH (Sec. III-D: the scene mesh with per-triangle      */
/* materials; the hierarchy is this library's own, 30-bit Morton codes,    */
/* radix sort, Karras hierarchy, bottom-up refit)                          */
/* ---------------------------------------------------------------------- */
/* vertices [n_vertices][3] float (metres), triangles [n_triangles][3] vertex
   indices, material_ids [n_triangles], materials [n_materials]; all host or
   device.  Triangles are wound so that (v1 - v0) x (v2 - v0) points out of
   their material.  Invalid indices, material ids or non-finite vertices give
   RR_ERR_INVALID_ARG.  The scene keeps its own copies; *out receives the
   handle.  Blocking. */
int rr_scene_create(const float* vertices, uint32_t n_vertices, const uint32_t* triangles, uint32_t n_triangles,
                    const uint16_t* material_ids, const rr_material* materials, uint32_t n_materials,
                    rr_scene** out);

/* Frees the scene and its workspace.  NULL is accepted. */
int rr_scene_destroy(rr_scene* scene);

/* New vertex positions [n_vertices][3] (host or device) for the same
   topology and materials; rebuilds the LBVH (Morton, sort, hierarchy,
   refit) without allocating.  Stream ordered; non-finite vertices give
   RR_ERR_INVALID_ARG at the next blocking call or rr_scene_sync. */
int rr_scene_update_vertices(rr_scene* scene, const float* vertices);

/* Sizes of the scene and its latest build.  Blocking (reads the wide node
   count of the latest build). */
int rr_scene_info_get(const rr_scene* scene, rr_scene_info* info);

/* Sets the lobe of material `material` (created with RR_MAT_TABULATED_LOBE)
   to the symmetric density given at RR_LOBE_SAMPLES points x_j = j (pi/2) /
   (RR_LOBE_SAMPLES - 1) of [0, pi/2] (host or device; finite, >= 0, not all
   zero).  The density between samples is the quadratic through each triple
   (x_2k, x_2k+1, x_2k+2); it is normalised to unit integral over
   [-pi/2, pi/2].  Rebuilds the scene's lobe tables (stream ordered). */
int rr_scene_set_lobe(rr_scene* scene, uint32_t material, const float* density);

/* Scene serialisation (no counterpart in the paper: a simulation saves the
   scene it scans and resumes from it later, or ships it to another process).
   rr_scene_save writes the scene's current state -- its vertices (as updated
   by rr_scene_update_vertices), triangles, material ids, materials, the
   densities of its tabulated lobes and its launch configuration
   (rr_batch_config, including the BVH build) -- into blob[capacity], host
   memory, behind a header with a format version and a checksum.  *size
   receives the bytes the blob takes; blob may be NULL to ask for it.
   RR_ERR_INVALID_ARG when capacity is too small (*size is still set).
   Blocking (waits for the scene's stream). */
int rr_scene_save(const rr_scene* scene, void* blob, uint64_t capacity, uint64_t* size);

/* Creates a scene from a blob written by rr_scene_save: the same mesh,
   materials, lobes and launch configuration.  The BVH is built again from
   them; the build is deterministic, so the new scene's hierarchy equals the
   saved scene's node for node and its scans give the same segments.
   RR_ERR_INVALID_ARG for a blob that is truncated, corrupted (checksum) or of
   another format version; otherwise as rr_scene_create.  Blocking. */
int rr_scene_load(const void* blob, uint64_t size, rr_scene** out);

/* Copies the LBVH to host arrays (each may be NULL): morton [T] sorted
   Morton codes, perm [T] triangle id of each sorted leaf, children
   [(T-1)][2] child references of the internal nodes (leaf j encoded as
   j | 0x80000000), parents [2T-1] parent of internal nodes 0..T-2 then of
   leaves (T-1)+j (root: RR_NO_HIT), boxes [(T-1)][2][6] child boxes of
   every internal node (lo xyz, hi xyz).  Blocking. */
int rr_scene_export_bvh(const rr_scene* scene, uint32_t* morton, uint32_t* perm, uint32_t* children,
                        uint32_t* parents, float* boxes);

/* Copies the 8-wide quantised BVH to host arrays (each may be NULL): nodes
   [n_wide_nodes][80 bytes] in the layout below and tris [T][3][4] float, the
   triangles in wide-leaf order (v0, v1, v2 with w = original triangle id,
   material id as bit patterns).  Node layout, five 16-byte words:
     w0 = P.x, P.y, P.z (float), ex | ey << 8 | ez << 16 | imask << 24
     w1 = first internal child, first triangle, valid slot mask, leaf
          triangle counts (2 bits per slot, slot k at bits 2k) (uint32)
     w2..w4 = child bounds as bytes: qlo.x[8], qlo.y[8], qlo.z[8], qhi.x[8],
              qhi.y[8], qhi.z[8]
   Slot k's bound on axis a is P.a + (2^23 + q) 2^(e_a - 127), an exact
   float; internal slots (imask) are children first_child + (number of
   internal slots below k); a leaf slot holds 1..3 consecutive triangles
   (this library's builder groups at most two) from first_triangle + (the
   triangle counts of the leaf slots below k).
   Node 0 is the root.  *n_nodes receives the node
   count; at most cap nodes are written.  The wide BVH is collapsed from the
   binary one when first needed after a build (a scan with RR_NODES_WIDE8 or
   this call).  Blocking. */
int rr_scene_export_wide(rr_scene* scene, void* nodes, uint32_t cap, uint32_t* n_nodes, float* tris);

/* ---------------------------------------------------------------------- */
/* scans                                                                   */
/* ---------------------------------------------------------------------- */
/* One polar image (Sec. III-A..C) for the pose: out_polar [n_azimuth][n_bins]
   float, host or device.  Blocking; returns the device status of the scan
   (RR_ERR_CAPACITY if the ray tree outgrew the workspace -- the message
   gives the size needed). */
int rr_scan(rr_scene* scene, const rr_pose* pose, const rr_sensor_params* params, float* out_polar);

/* Same, non-blocking: out_polar must be device memory; returns after the
   kernels are queued.  Device-side errors are reported by rr_scene_sync. */
int rr_scan_async(rr_scene* scene, const rr_pose* pose, const rr_sensor_params* params, float* out_polar);

/* Waits for the scene's queued work and returns (then clears) the sticky
   device status of the scans and rebuilds since the previous sync. */
int rr_scene_sync(rr_scene* scene);

/* n scans of one scene, each with its own pose and sensor model (ray counts,
   bounce limits, bins and flags may all differ): poses [n], params [n],
   out [n] pointers to images (host or device, each
   [params[i].n_azimuth][params[i].n_bins]).  The scans are traced together:
   consecutive scans whose worst-case ray trees fit the workspace limit
   (rr_batch_config) share one launch sequence -- ray generation, the
   trace/shade wavefront of every bounce and the image pass -- so small scans
   fill the GPU together.  Each image equals the scan run alone up to the
   rounding of the float sums (the order in which returns are added to a bin
   is not fixed).  Blocking; returns the device status of the batch. */
int rr_scan_batch(rr_scene* scene, uint32_t n, const rr_pose* poses, const rr_sensor_params* params,
                  float* const* out);

/* Same, non-blocking: every out[i] must be device memory; returns once the
   work is queued.  Device-side errors are reported by rr_scene_sync. */
int rr_scan_batch_async(rr_scene* scene, uint32_t n, const rr_pose* poses, const rr_sensor_params* params,
                        float* const* out);

/* Launch parameters of the batched path (per scene).  The paper has no
   counterpart; they trade memory and occupancy for throughput only and never
   change a result beyond float summation order.
   wavefront_rays       most initial rays traced in one launch sequence
                        (0: as many as the workspace limit allows)
   trace_block          threads per block of the trace kernel: 64, 128 or 256
   trace_blocks_per_sm  resident trace blocks per SM (0: the occupancy maximum)
   use_graph            1: each launch sequence is captured once in a CUDA
                        graph and replayed while its arguments stay the same
   node_format          RR_NODES_BINARY (default): traverse the binary LBVH
                        with float boxes; RR_NODES_WIDE8: the 8-wide BVH with
                        8-bit quantised child boxes.  Both give the same
                        closest hit for every query (the quantised boxes are
                        rounded outward onto exact float bounds).
   refill_threshold     the query kernels keep their lanes busy by handing a
                        warp's idle lanes new queries once at least this many
                        of its 32 lanes are idle (1..32; 0 = 16)
   workspace_limit      bytes of scan workspace; a launch sequence is sized
                        for its worst-case ray tree (every hit spawning both
                        children) within this limit (0: 24 GiB)
   split_streams        rr_scan / rr_scan_async trace a scan as this many
                        azimuth ranges, each on its own stream, so that the
                        slow queries closing one range's bounce overlap the
                        other ranges' work (1..4; 0: the default, 3).  Scans
                        with a beam pattern run whole.  The image is the same
                        up to the rounding of the bin sums.
   bvh_build            RR_BVH_SAH_TOP (default): the LBVH (Morton codes,
                        radix sort, Karras hierarchy, refit) with the part
                        above its subtrees of at most 32 triangles rebuilt
                        top down by binned SAH over those subtrees (HLBVH);
                        RR_BVH_LBVH: the LBVH alone.  Every build of the
                        scene (creation, rr_scene_update_vertices) uses it;
                        setting a different value rebuilds the BVH (blocking).
                        Both give the same closest hit for every query; the
                        SAH top needs fewer node visits.
   query_order          order in which the closest-hit queries of bounces >= 1
                        are handed to the query kernel: RR_ORDER_QUEUE (the
                        queue order: children of neighbouring rays together,
                        reflected and refracted interleaved) or
                        RR_ORDER_CELL_OCTANT (bucketed by the ray's direction
                        octant and a cell of its origin around the sensor, so
                        that the lanes of a warp trace rays that go the same
                        way from the same region).  Every query's result is
                        the same in either order. */
#define RR_NODES_WIDE8 0u
#define RR_NODES_BINARY 1u
#define RR_BVH_LBVH 0u
#define RR_BVH_SAH_TOP 1u
#define RR_ORDER_QUEUE 0u
#define RR_ORDER_CELL_OCTANT 1u
typedef struct {
  uint32_t wavefront_rays;
  uint32_t trace_block;
  uint32_t trace_blocks_per_sm;
  uint32_t use_graph;
  uint32_t node_format;
  uint32_t refill_threshold;
  uint64_t workspace_limit;
  uint32_t split_streams;
  uint32_t bvh_build;
  uint32_t query_order;
  uint32_t reserved;
} rr_batch_config;

int rr_batch_config_get(const rr_scene* scene, rr_batch_config* out);
/* RR_ERR_INVALID_ARG for a trace_block other than 64/128/256, more than 64
   blocks per SM, use_graph > 1, an unknown node_format or bvh_build, a
   refill_threshold above 32, split_streams above 4, an unknown query_order
   (reserved must be 0) or a workspace limit
   below 1 MiB. */
int rr_batch_config_set(rr_scene* scene, const rr_batch_config* config);

/* How rr_scan_batch would cut scans params[0..n) into launch sequences under
   config (NULL: the defaults), computed on the host only (no device work,
   usable without a GPU).  first [cap] receives the index of each sequence's
   first scan (a sequence runs to the next one's first scan), *n_groups the
   number of sequences (only min(cap, *n_groups) entries are written) and
   *max_workspace the workspace bytes of the largest sequence.  A sequence
   holds at most 65535 scans, 2^18 azimuth columns, 2^30 initial rays and
   fewer than 2^32 pixels of beam-pattern images,
   at most wavefront_rays initial rays and a worst-case workspace within
   workspace_limit, except a single scan, which is sized down to the limit
   (and may then report RR_ERR_CAPACITY when it runs). */
int rr_batch_plan(uint32_t n, const rr_sensor_params* params, const rr_batch_config* config, uint32_t* first,
                  uint32_t cap, uint32_t* n_groups, uint64_t* max_workspace);

/* Autotuner: runs the batch (poses, params as for rr_scan_batch, images kept
   on the device and discarded) under a sequence of launch configurations --
   node format, then wavefront size, then trace block size, then trace blocks
   per SM, then the refill threshold, then graph replay, keeping the best of
   each -- each timed with CUDA events as
   the mean of reps passes after one warm-up pass.  Sets the fastest on the
   scene and returns it in *best (may be NULL) with its time in *best_ms and
   the time of the configuration it started from in *start_ms (each may be
   NULL).  Blocking; allocates the images of one pass. */
int rr_autotune(rr_scene* scene, uint32_t n, const rr_pose* poses, const rr_sensor_params* params, uint32_t reps,
                rr_batch_config* best, float* best_ms, float* start_ms);

/* Debug scan: like rr_scan, plus
   ray_mask  [n_azimuth * rays_per_beam] uint8 or NULL; initial rays with a
             non-zero mask are traced but add nothing to the image
   segs      [seg_capacity] segment records (NULL: none); *n_segs receives the
             number of segments traced (may exceed seg_capacity, then
             RR_ERR_CAPACITY and only seg_capacity records are written)
   ray_tallies [n_azimuth * rays_per_beam][4] float or NULL: per initial ray
             the energy returned, absorbed, escaped and terminated
   All buffers host or device.  Segments are ordered by bounce, then by
   queue position.  Blocking. */
int rr_scan_debug(rr_scene* scene, const rr_pose* pose, const rr_sensor_params* params, const uint8_t* ray_mask,
                  float* out_polar, rr_segment* segs, uint64_t seg_capacity, uint64_t* n_segs, float* ray_tallies);

/* Same scan as rr_scan, for callers that cannot allocate device memory
   while they run: real-time loops that must never block on the allocator
   (cudaMalloc / cudaFree can synchronise the device) and programs whose device
   memory belongs to another allocator under a fixed budget.  The paper has no
   counterpart; this is a property of the library, not of the method.
   Allocates nothing: the scan's scratch (ray queues, hits, return records,
   tile flags) lives in one fixed 64 MiB device array compiled into the
   library, which every GPU that loads the library holds until the process
   exits.  The scene (created beforehand with rr_scene_create) and out_polar
   [n_azimuth][n_bins] (device memory) are the caller's.  A scan whose
   worst-case scratch exceeds 64 MiB is rejected with RR_ERR_INVALID_ARG and a
   message giving the size; the 400 x 8 ray, 3 bounce, 1142 bin tiny room
   needs about 4 MiB.  The first call on each device, with that device current,
   looks up the array's device address once.  All calls share the array
   (it keeps the last call's contents; the scan writes everything before it
   reads it), so calls that overlap on the GPU race; a call also shares the
   scene's status counters with rr_scan, so it must not overlap any other
   scan of the same scene either.  It always traverses the binary BVH (the
   same closest hits as the 8-wide one, without its lazy collapse), whatever
   node format rr_batch_config_set chose.  The scene must live on the
   current device (else RR_ERR_INVALID_ARG).  Blocking; returns the device
   status of the scan. */
int rr_scan_static(rr_scene* scene, const rr_pose* pose, const rr_sensor_params* params, float* out_polar);

/* Range-bin accumulation alone (Sec. III-B): the image pass of a scan run on
   caller-given returns.  Return k adds energy[k] to pixel (column[k],
   bin[k]) of out [n_columns][n_bins]; there is no blur, pattern or noise.
   The sums are FP32 with compensated (Neumaier) summation, the same kernel as
   in every scan.  column [n] must be non-decreasing and below n_columns (else
   RR_ERR_INVALID_ARG); returns with bin >= n_bins are dropped; n_columns <=
   2^18, n_bins <= 16384.
   All buffers host or device.  Blocking. */
int rr_accumulate_returns(const uint32_t* column, const uint32_t* bin, const float* energy, uint64_t n,
                          uint32_t n_columns, uint32_t n_bins, float* out);

/* Sec. III-B display mapping: L_E = 10 log10(E_R / E0), E0 = 1, mapped
   linearly from [-cutoff_db, 0] dB to [0, 255], clamped, rounded to nearest.
   polar [n] float and out [n] uint8 are device memory.  Stream ordered. */
int rr_polar_to_db_u8(const float* polar, uint64_t n, float cutoff_db, uint8_t* out);

/* ---------------------------------------------------------------------- */
/* serving: resident scenes, requests from many clients, continuous        */
/* batching (the paper has no counterpart; it serves the same scans)       */
/* ---------------------------------------------------------------------- */
typedef struct rr_server rr_server; /* opaque */

/* memory_budget    device bytes the server holds for work in flight, split
                    evenly into one fixed arena per slot when the server is
                    created (0: 16 GiB); nothing is allocated while serving
   slots            launch sequences in flight at once, each on its own
                    stream (1..16; 0: 4)
   max_batch_scans  most requests per launch sequence (0: 64)
   max_batch_rays   most initial rays per launch sequence (0: 4 Mi); a
                    single larger request still runs alone
   max_queue        most requests waiting for a slot (0: 4096); beyond it
                    rr_serve_submit returns RR_ERR_BUSY
   node_format, refill_threshold   as in rr_batch_config
   admission        RR_ADMIT_ESTIMATE (default): a batch's workspace is sized
                    by an estimate of its ray tree -- the largest queue and
                    return counts per initial ray seen at every bounce of
                    the scene's earlier batches (bounces not seen yet: twice
                    the previous bounce), times estimate_factor; the scene's
                    first batch, and any batch that outgrows its estimate
                    (rerun, never dropped: rr_serve_stats.retried), are sized
                    for the worst case.  RR_ADMIT_WORST_CASE: always the
                    worst case (every hit spawning both children).
   estimate_factor  safety factor of the estimate (0: 2; must be >= 0) */
#define RR_ADMIT_ESTIMATE 0u
#define RR_ADMIT_WORST_CASE 1u
typedef struct {
  uint64_t memory_budget;
  uint32_t slots;
  uint32_t max_batch_scans;
  uint32_t max_batch_rays;
  uint32_t max_queue;
  uint32_t node_format;
  uint32_t refill_threshold;
  uint32_t admission;
  float estimate_factor;
} rr_serve_config;

/* request states */
#define RR_REQ_QUEUED 0
#define RR_REQ_RUNNING 1
#define RR_REQ_DONE 2
#define RR_REQ_FAILED 3
#define RR_REQ_CANCELLED 4   /* cancelled while queued: it never ran, out_polar untouched */

/* One request: state, status (RR_OK or the failure), times in ms of the
   host steady clock since the server was created: submitted, launched,
   completed (observed by the server), and the number of requests of the
   launch sequence it ran in. */
typedef struct {
  int32_t state;
  int32_t status;
  double submit_ms, start_ms, done_ms;
  uint32_t batch_size;
  uint32_t reserved;
} rr_serve_record;

/* Since the last reset: requests submitted / completed / failed / refused
   (queue full), launch sequences, closest-hit and visibility queries traced,
   initial rays, wall time with work in flight (busy_ms) and elapsed, the
   requests still queued, and the latency (submit to completion) of the
   completed requests: median, 99th percentile (nearest rank), mean, max. */
typedef struct {
  uint64_t submitted, completed, failed, rejected_busy;
  uint64_t batches, closest_queries, anyhit_queries, initial_rays;
  uint64_t queued;
  double busy_ms, elapsed_ms;
  double latency_p50_ms, latency_p99_ms, latency_mean_ms, latency_max_ms;
  uint64_t retried;   /* requests rerun at worst-case size after their estimated batch overflowed */
  uint64_t cancelled; /* requests cancelled while queued (rr_serve_cancel) */
} rr_serve_stats;

/* Starts a server (its worker thread and slots) on the current device.
   config may be NULL (all defaults).  Scenes are the caller's: they must stay
   alive, and unchanged, while requests on them are unfinished. */
int rr_serve_create(const rr_serve_config* config, rr_server** out);

/* Finishes the requests already submitted, then frees the server.  Records
   not yet read are lost.  NULL is accepted. */
int rr_serve_destroy(rr_server* server);

/* Queues one scan (the same as rr_scan of the scene with pose and params)
   writing out_polar [n_azimuth][n_bins] (host or device; it must stay valid
   until the request finishes).  Returns at once with a ticket.
   RR_ERR_INVALID_ARG for bad parameters or a request whose worst-case scratch
   exceeds a slot's arena, RR_ERR_BUSY when the queue is full. */
int rr_serve_submit(rr_server* server, rr_scene* scene, const rr_pose* pose, const rr_sensor_params* params,
                    float* out_polar, uint64_t* ticket);

/* *done = 1 once the request has finished (completed or failed), else 0.
   Non-blocking. */
int rr_serve_poll(rr_server* server, uint64_t ticket, int* done);

/* Waits up to timeout_ms for the request; returns its status (RR_OK when it
   completed), or RR_ERR_TIMEOUT if it is still unfinished. */
int rr_serve_wait(rr_server* server, uint64_t ticket, uint32_t timeout_ms);

/* The request's record; a finished request's ticket is then forgotten. */
int rr_serve_result(rr_server* server, uint64_t ticket, rr_serve_record* out);

/* Cancels a request that is still queued: it never runs, its out_polar is
   not written, and it finishes at once as RR_REQ_CANCELLED (rr_serve_wait
   returns RR_ERR_CANCELLED; its record can be read as for any finished
   request).  *cancelled = 1 then.  A request already launched (its batch
   is on the GPU) or finished is left as it is, *cancelled = 0: a launched
   batch is not interrupted, and its outputs are written.  A request queued
   again to rerun at worst-case size is queued and can be cancelled.
   RR_ERR_INVALID_ARG for an unknown ticket.  Non-blocking.  (No counterpart
   in the paper: serving clients such as robots that move on abandon scans
   they no longer need.) */
int rr_serve_cancel(rr_server* server, uint64_t ticket, int* cancelled);

/* Server statistics (see rr_serve_stats); reset != 0 starts a new window. */
int rr_serve_stats_get(rr_server* server, rr_serve_stats* out, int reset);

/* ---------------------------------------------------------------------- */
/* counters                                                                */
/* ---------------------------------------------------------------------- */
/* Cumulative query counters of the scene (blocking); reset != 0 clears them. */
int rr_scene_stats(rr_scene* scene, rr_stats* stats, int reset);

/* Per-kernel device time with CUDA events on the scene's launches.  While
   enabled, each launch is bracketed by two events on its stream; the events
   are placed on one time line by a base event recorded on the calling
   thread's stream when profiling is switched on. */
int rr_profile_enable(rr_scene* scene, int on);
int rr_profile_read(rr_scene* scene, rr_profile* out, int reset);

#ifdef __cplusplus
}
#endif
#endif /* RR_H */

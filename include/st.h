/*
 * st.h -- C ABI of the GB300 differentiable path tracer (libst.so).
 *
 * The library renders a triangle mesh with per-face Torrance-Sparrow
 * reflectance under point lights and/or an HDR environment map by Monte Carlo
 * path tracing, and computes the gradient of an image loss with respect to the
 * vertex positions and the per-face material parameters. This is the
 * differentiable renderer R(x, m, c) the paper optimises through (Sec. 3.2,
 * "Vertex optimization": the MSE loss over views c_i and its gradient with
 * respect to vertex positions x; Sec. 3.3, "Material Optimization": the same
 * loss with respect to the material m; material "Representation": a
 * Torrance-Sparrow BRDF with diffuse albedo, specular and roughness per mesh
 * facet, i.e. mesh colors at resolution r = 0; Sec. 3.1 "Input": point lights
 * or an HDR environment map; Sec. 3.3 "Effects of Global Illumination":
 * multi-bounce transport, max_bounces = 1 being "local + shadows").
 *
 * Conventions shared by every call:
 *  - Every call returns an st_status; nothing aborts. On a non-OK status,
 *    st_last_error() gives a message (thread-local, valid until the next call
 *    on the same thread).
 *  - Device pointers are CUDA device memory of the device that is current when
 *    the scene was created; they are owned by the caller unless stated.
 *    Host pointers are read before the call returns.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream). Calls enqueue
 *    work and return without synchronising unless stated; outputs are valid
 *    when the stream reaches that point.
 *  - A scene is not thread-safe; distinct scenes are independent. Calls on one
 *    scene must be issued on one stream, or ordered by the caller.
 *  - Images are packed: view v occupies rows [pixel_offset, pixel_offset+W*H)
 *    of a float [N][3] array, row-major within the view, row 0 at the top.
 *  - Randomness is a pure function of (seed, view pixel_offset, pixel,
 *    sample): identical arguments give a bitwise identical image whatever
 *    the batching mode; st_render_backward with the same seed replays the
 *    forward paths (no path storage between the two calls).
 */
#ifndef ST_H
#define ST_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ST_OK = 0,
  ST_ERR_INVALID_ARG = 1,  /* a size, pointer or index is out of range */
  ST_ERR_OOM = 2,          /* device or host allocation failed */
  ST_ERR_CUDA = 3,         /* a CUDA runtime call failed (message has the CUDA error) */
  ST_ERR_TIMEOUT = 4,      /* reserved: no call in this library waits on a device flag */
  ST_ERR_STATE = 5,        /* call not valid for the scene's current state */
  ST_ERR_UNSUPPORTED = 6,  /* feature outside the library's limits (see ST_MAX_*) */
  ST_ERR_DEVICE = 7        /* a kernel latched an error (e.g. BVH stack overflow) */
} st_status;

#define ST_MAX_LIGHTS 8
#define ST_MAX_BOUNCES 8
#define ST_BRDF_GGX 0
#define ST_BRDF_BECKMANN 1
#define ST_EDGE_SILHOUETTE 0  /* edges whose two faces face opposite ways, and boundary edges */
#define ST_EDGE_ALL 1         /* every mesh edge (also the shading discontinuities of flat faces) */
#define ST_FRESNEL_HELD 0      /* st_scene_desc.fresnel: specular lobe scaled by ks at every angle */
#define ST_FRESNEL_SCHLICK 1   /* st_scene_desc.fresnel: Schlick's Fresnel factor with F0 = ks */
#define ST_BVH_PLOC 0   /* tree by locally-ordered clustering (Meister and Bittner 2018): lower traversal cost */
#define ST_BVH_LBVH 1   /* Karras radix tree over the Morton order: faster build */
#define ST_EDGE_TERM_PRIMARY 1    /* edge_term bit: primary visibility (image-space edges) */
#define ST_EDGE_TERM_SECONDARY 2  /* edge_term bit: secondary visibility (edges seen from path vertices) */
#define ST_EDGE_TERM_SHADOW 4     /* edge_term bit: point-light shadow boundaries on surfaces the camera sees */
#define ST_MODE_BATCHED 0     /* all views in one job space, persistent kernels, optional CUDA graph */
#define ST_MODE_PER_VIEW 1    /* one view at a time, grids sized from host-read queue counts */

typedef struct st_scene st_scene; /* opaque, library-owned */

/* Point light (Sec. 3.1): position and radiant intensity (W/sr), RGB. */
typedef struct {
  float pos[3];
  float intensity[3];
} st_point_light;

/* Equirectangular HDR environment (Sec. 3.1 "Input": an HDR environment map
 * as the light): rgb = float [H][W][3] radiance in device memory of the
 * current device or in host memory (st_scene_create tells them apart with
 * cudaPointerGetAttributes; device memory is read back once, since the alias
 * table is built on the host). Row 0 is theta = 0 (the +y pole); direction for
 * (theta, phi) is (-sin theta sin phi, cos theta, sin theta cos phi),
 * phi = 2 pi (col + 0.5)/W at texel centres. Copied, and its FP64 alias table
 * built, at scene create; the caller keeps ownership. */
typedef struct {
  int width, height;
  const float* rgb;
} st_envmap;

/* Pinhole view c_i (Sec. 3.2): fov_y in degrees, +y up on screen. spp == 0
 * takes the call's default_spp. pixel_offset = first packed-image row of the
 * view; it also keys the view's random numbers. lights: point lights that
 * only this view's paths see, after the scene's (the paper lights each capture
 * from the camera and from a point offset from it, Sec. 4); the scene's and
 * the view's lights together are at most ST_MAX_LIGHTS. */
#define ST_MAX_VIEW_LIGHTS 2
#define ST_MAX_VIEWS 65535        /* views per call (and, for the shadow-edge term, (view, light) pairs) */
#define ST_SEC_PICK_TREE 0        /* st_render_opts.sec_pick: importance through the edge hierarchy */
#define ST_SEC_PICK_UNIFORM 1     /* st_render_opts.sec_pick: uniform over all edges */
typedef struct {
  float eye[3], target[3], up[3];
  float fov_y_deg;
  int width, height, spp;
  long long pixel_offset;
  int n_lights;                                     /* 0..ST_MAX_VIEW_LIGHTS */
  struct { float pos[3]; float intensity[3]; } lights[ST_MAX_VIEW_LIGHTS];
} st_view;

/* Material: mesh colors (Sec. 3.3) at resolution r = color_res. Face t owns
 * the texels t*n .. t*n + n - 1, n = (r+1)(r+2)/2; a point of barycentric
 * weights (alpha, beta) for the face's second and third vertices uses texel
 * k = (t (r+1)(r+2) + i (2r - i + 3)) / 2 + j, (i, j) = floor(r (alpha, beta)).
 * r = 0 is one parameter set per face. Each texel holds kd_r, kd_g, kd_b, ks,
 * roughness (or, with rgb_specular, kd_r, kd_g, kd_b, ks_r, ks_g, ks_b,
 * roughness: the paper's "specular color", Sec. 3.3). */
typedef struct {
  int n_vertices, n_faces;
  const float* vertices;     /* device, float [V][3] */
  const int* faces;          /* device, int [F][3] vertex indices */
  const float* face_params;  /* device, float [F*n][5 or 7] texel parameters (n = 1 when color_res = 0) */
  int brdf;                  /* ST_BRDF_GGX or ST_BRDF_BECKMANN */
  int n_point_lights;        /* 0..ST_MAX_LIGHTS (a call needs some light: these, the environment or its views') */
  const st_point_light* point_lights; /* host array */
  const st_envmap* env;      /* NULL if no environment */
  int color_res;             /* mesh-colors resolution r, 0..64 */
  int bvh_builder;           /* ST_BVH_PLOC (0, default) or ST_BVH_LBVH; st_scene_create and st_rebuild use it */
  int rgb_specular;          /* 0: 5 parameters per texel (kd rgb, ks, roughness); 1: 7 (kd rgb, ks rgb,
                                roughness), a specular colour per channel. face_params, st_set_face_params and
                                the d_face_params of st_render_backward all use this layout. */
  int smooth_normals;        /* 0: flat face normals (the paper's facets). 1: shading normals interpolated from
                                vertex normals: N_v = normalised sum of (v1 - v0) x (v2 - v0) over the faces
                                around v (recomputed after every vertex update); at a hit of barycentric weights
                                (b1, b2), n_s = normalise((1 - b1 - b2) N0 + b1 N1 + b2 N2), turned with the face
                                normal toward the incoming ray. Lights, environment samples and sampled
                                directions count only above both the face's and the shading plane. Gradients
                                reach every vertex around a hit face. */
  int fresnel;               /* Fresnel factor of the Torrance-Sparrow specular lobe (Sec. 3.3
                                "Representation"): ST_FRESNEL_HELD (0, default) keeps it at ks at every angle,
                                so ks = 0 is exactly Lambertian; ST_FRESNEL_SCHLICK (1) takes Schlick's
                                approximation with F0 = ks per channel, F = ks + (1 - ks)(1 - wi.h)^5, h the
                                half vector. Sampling (lobe probability, pdfs) is the same in both. */
} st_scene_desc;

typedef struct {
  int edge_term;    /* backward: OR of ST_EDGE_TERM_PRIMARY, _SECONDARY and _SHADOW (0 = interior only) */
  int edge_mode;    /* ST_EDGE_SILHOUETTE or ST_EDGE_ALL (silhouettes as seen from the camera, or from each
                       path vertex for the secondary term) */
  int edge_spp;     /* edge samples per pixel; 0 = the view's spp */
  int mode;         /* ST_MODE_BATCHED or ST_MODE_PER_VIEW */
  int use_graph;    /* batched mode: capture and replay the call as a CUDA graph */
  int chunk_paths;  /* paths in flight per wavefront chunk; 0 = library default */
  int time_kernels; /* per-view or ungraphed batched: time the closest-hit and any-hit kernels and the GPU-side
                       intervals between host synchronisations (see st_stats) */
  int count_visits; /* run the instrumented traversal that counts node visits and triangle tests */
  int persist_blocks; /* batched mode: resident blocks per SM of the persistent stage kernels (0 = occupancy limit) */
  unsigned long long* path_signatures; /* forward, optional: device uint64 [N], same rows as out_image: per pixel,
                       the sum over its samples (mod 2^64) of a 64-bit FNV-1a hash of each path's discrete decisions:
                       at every vertex the face hit (0xffffffff for a miss), then for a miss under an environment
                       the texel its direction reads, for a hit with mesh colors at r > 0 the texel it picks,
                       the environment texel drawn for NEE,
                       the BSDF lobe code (1 = specular, + 2 when the direction is valid) where one is drawn, then
                       the shadow rays' visibility bits (bit j = point light j seen, bit 8 = the environment sample
                       seen) when any was traced; basis 0xcbf29ce484222325, prime 0x100000001b3. Equal signatures
                       with another implementation of the estimator mean the same decisions were taken. */
  int sec_pick;     /* backward, secondary edge term: how each path vertex picks its edge. ST_SEC_PICK_TREE (0,
                       default): through a hierarchy over the edges (Li et al. sample secondary edges by
                       importance, Sec. 3.2): blocks of consecutive edges (at most 2^14) under a binary tree of
                       boxes and summed lengths; a node weighs 0 below the vertex's tangent plane, else its length
                       over max(d^2, diag^2/4); one uniform per level, uniform within the block; the sample is
                       divided by its probability. ST_SEC_PICK_UNIFORM: one edge uniformly from all. */
} st_render_opts;

typedef struct {
  long long paths;            /* camera + edge-side paths started by the last call */
  long long extension_rays;   /* closest-hit queries of the last call */
  long long shadow_rays;      /* any-hit queries of the last call */
  long long edge_samples;     /* edge samples of the last call (each traces two paths) */
  long long node_visits;      /* instrumented calls only: internal nodes fetched by closest-hit */
  long long tri_tests;        /* instrumented calls only: triangle tests by closest-hit */
  int extend_launches;        /* closest-hit launches timed (time_kernels): ray generation, which finds the hits of
                                 the first rays a screen-space bin serves, and the BVH traversals */
  double extend_ms;           /* their summed CUDA-event time */
  int device_error;           /* latched device error bits (0 = none) */
  int bvh_nodes;              /* internal nodes of the binary BVH (refit / st_debug_bvh layout) */
  long long scratch_bytes;    /* device bytes held by the scene's wavefront buffers */
  int kernel_launches;        /* kernels the last call launched (graph kernel nodes included) */
  int bvh4_nodes;             /* nodes of the 4-wide BVH the traversal walks */
  long long secondary_samples; /* accepted secondary edge samples of the last call (each traces two paths) */
  long long shadow_node_visits; /* instrumented calls only: internal nodes fetched by any-hit (shadow) queries */
  long long shadow_tri_tests;   /* instrumented calls only: triangle tests by any-hit queries */
  int shadow_launches;        /* any-hit launches timed (time_kernels) */
  double shadow_ms;           /* their summed CUDA-event time */
  double busy_ms;             /* time_kernels: GPU time of the call between its host synchronisations (a per-view
                                 call reads queue counts back; the rest of its wall time the GPU waits on the host) */
  int host_syncs;             /* host synchronisations of the last call (per-view mode reads queue counts back) */
} st_stats;

/* Create a scene from the reconstruction's state (Sec. 3.1 "Input": a
 * triangle mesh of vertex positions x, lit by point lights or an HDR
 * environment map; Sec. 3.3 "Representation": a Torrance-Sparrow material per
 * facet, or mesh colors at resolution r). Copies the mesh and the texel
 * parameters into scene-owned device memory, checks them on the host (face
 * indices in range, no repeated index in a face, finite vertices, lights and
 * environment valid), builds the BVH (Morton codes, radix sort, then PLOC
 * clustering or Karras' radix tree, bottom-up boxes, 4-wide collapse), the edge
 * list and the environment's FP64 alias table. *out receives the handle, owned
 * by the library until st_scene_destroy. Errors: ST_ERR_INVALID_ARG (bad
 * description), ST_ERR_UNSUPPORTED (beyond the limits), ST_ERR_OOM (device
 * memory), ST_ERR_CUDA; on any error *out is NULL and nothing is held.
 * Synchronises `stream`. */
st_status st_scene_create(const st_scene_desc* desc, void* stream, st_scene** out);

/* Free everything the scene owns. NULL is accepted. */
st_status st_scene_destroy(st_scene* scene);

/* New vertex positions (device float [V][3], same topology): recompute
 * triangle records and boxes bottom-up on the existing hierarchy. The vertex
 * update of every optimisation step (Sec. 3.2). */
st_status st_refit(st_scene* scene, const float* new_vertices, void* stream);

/* New vertex positions with a full rebuild (Morton order recomputed). */
st_status st_rebuild(st_scene* scene, const float* new_vertices, void* stream);

/* New texel parameters (device float [F*n][5 or 7], see st_scene_desc); the material update (Sec. 3.3). */
st_status st_set_face_params(st_scene* scene, const float* face_params, void* stream);

/* The renderer R(x, m, c_i) of the paper's loss (Sec. 3.2 "Vertex
 * optimization": the images of the current reconstruction seen from the
 * cameras c_i; Sec. 3.3 "Effects of Global Illumination": multi-bounce
 * transport). Monte Carlo forward render of n_views views (host array,
 * 1..ST_MAX_VIEWS) with max_bounces surface vertices per path
 * (1..ST_MAX_BOUNCES). out_image: caller-owned device float [N][3], N = max
 * over views of pixel_offset + W*H, row-major per view; it is overwritten on
 * every pixel of the views (other rows untouched). opts may be NULL (batched,
 * graph on). Asynchronous on `stream`. Errors: ST_ERR_INVALID_ARG (bad views,
 * overlapping pixel ranges, no light), ST_ERR_UNSUPPORTED, ST_ERR_OOM, ST_ERR_CUDA;
 * a kernel's latched error is reported by st_get_stats (device_error).
 * A call of at least 2^20 primary rays finds their hits in screen-space leaf
 * lists of its views, kept on the device: a later call (forward or backward)
 * with the same views (camera, size) and no vertex update since uses them
 * without building them again. Such a call also bins the leaves, seen from each
 * scene light outside the mesh's bounding sphere, into a frustum of cells, and
 * the shadow rays to that light test their cell's leaves instead of traversing
 * the BVH (the same test: the same visibility); these lists are rebuilt after a
 * vertex update. */
st_status st_render(st_scene* scene, const st_view* views, int n_views, int default_spp,
                    int max_bounces, unsigned long long seed, const st_render_opts* opts,
                    float* out_image, void* stream);

/* The gradient the paper descends (Sec. 3.2 "Vertex optimization": the loss
 * over the views c_i differentiated with respect to the vertex positions x,
 * through Li et al.'s edge sampling for visibility; Sec. 3.3 "Material
 * Optimization": the same loss with respect to the material). The loss itself
 * stays with the caller, who passes dL/dI. Errors as st_render.
 * Adjoint: given dL/dI (device float [N][3], same layout as out_image),
 * ACCUMULATE (+=) dL/dvertices into d_vertices (device float [V][3]) and
 * dL/dtexel-parameters into d_face_params (device float [F*n][5 or 7], as the scene's layout). The interior term
 * replays the forward paths of the same seed and sweeps each in reverse; the
 * edge term (opts->edge_term) samples visibility edges: in screen space
 * (primary) and, at every vertex of every camera path, on the vertex's sphere
 * of directions (secondary: one uniformly picked mesh edge per vertex, two
 * side paths continuing from the next vertex), and, for every point light of
 * every view, along the image of the light's shadow boundary on the surfaces
 * the camera sees (shadow: an edge that is a silhouette seen from the light, a
 * point on it, the light ray through it continued to the receiving surface,
 * camera paths on both sides of that point's image). Either gradient pointer may be
 * NULL to skip it (d_vertices may not be NULL with edge_term). */
st_status st_render_backward(st_scene* scene, const st_view* views, int n_views, int default_spp,
                             int max_bounces, unsigned long long seed, const st_render_opts* opts,
                             const float* dL_dimage, float* d_vertices, float* d_face_params,
                             void* stream);

/* Closest-hit query through the BVH for n rays: rays device float [n][8] =
 * (ox, oy, oz, unused, dx, dy, dz, tmax), d of unit length; out_tri device
 * int [n] (face id, -1 = miss), out_t device float [n] (+inf on a miss). Hits
 * at t <= 1e-5 are not reported (the path tracer's self-intersection bound);
 * exclude_face is skipped (-1 = none); equal t resolves to the lower face id. */
st_status st_trace_closest(st_scene* scene, const float* rays, int n, int exclude_face, int* out_tri,
                           float* out_t, void* stream);

/* Statistics of the last render/backward call; synchronises the scene's work. */
st_status st_get_stats(st_scene* scene, st_stats* out);

/* Copy the BVH for inspection (host arrays, sizes from st_get_stats):
 * nodes float [F-1][16] as stored on the device, leaf_faces int [F]. */
st_status st_debug_bvh(st_scene* scene, float* nodes, int* leaf_faces);

/* Allocation-free BVH build, for callers that cannot allocate device memory
 * when they need one (an allocator at its budget, a framework that forbids
 * allocation on its hot path, an embedding that owns every buffer). The paper
 * has no counterpart: this is a library-side convenience. It runs the same
 * build as st_scene_create with bvh_builder = ST_BVH_LBVH (Morton order, radix
 * sort, Karras hierarchy, bottom-up boxes) and writes the same node and leaf
 * layout, but takes all
 * scratch from one fixed file-scope device array (about 1.8 MiB, held by every
 * device that loads the library until the process exits) and calls no
 * allocator. Inputs: vertices device float [V][3], faces device int [F][3].
 * Outputs (caller-owned, 16-byte aligned): nodes device float [F-1][16] (may
 * be NULL when F == 1), tris device float [F][12] (leaf triangle records),
 * leaf_faces device int [F] (face id of each leaf, Morton order).
 * Limits and behaviour:
 *  - F <= 65536, else ST_ERR_UNSUPPORTED; face indices are checked on the
 *    device first (ST_ERR_INVALID_ARG), and the build's device error word is
 *    read back at the end (ST_ERR_DEVICE when the bottom-up pass found a
 *    malformed tree): each call synchronises `stream` twice.
 *  - The first call on a device looks up the scratch array's device address
 *    (cudaGetSymbolAddress); make that first call before any stream capture.
 *  - Every call shares the one scratch array: calls that overlap on the GPU
 *    (other streams, other threads) race and corrupt each other's result. */
st_status st_build_bvh_noalloc(const float* vertices, const int* faces, int n_vertices, int n_faces,
                               float* nodes, float* tris, int* leaf_faces, void* stream);

/* Measurement utility, not part of the method: read bandwidth (GB/s) of a
 * device buffer of `bytes` (>= 1 MiB) that is resident in L2, read `passes`
 * times by one kernel with cache-global 16-byte loads. Allocates and frees the
 * buffer; synchronises `stream`. Used as the L2 roofline denominator. */
st_status st_measure_l2_read(long long bytes, int passes, void* stream, double* gbs);

/* Host-side fault injection, for testing how callers handle failures; the
 * paper has no counterpart. The nth next event (nth = 0: the next one) at
 * `site` fails as the CUDA call would have, without making that call:
 *  - ST_FAULT_ALLOC: a device allocation by the library (scene buffers,
 *    wavefront buffers, per-call tables). The call returns ST_ERR_OOM.
 *  - ST_FAULT_COPY: a copy between host and device of scene, call or
 *    statistics data. The call returns ST_ERR_CUDA.
 * nth < 0 disarms the site. Nothing is injected on the device. A call that
 * fails this way leaves its scene valid: later calls succeed, and
 * st_scene_destroy frees everything. The setting is process-wide (all
 * threads, all scenes). The library's first fault query also reads the
 * environment variable ST_FAULT ("alloc:N" or "copy:N"), for processes that
 * cannot call this function. Unknown site: ST_ERR_INVALID_ARG. */
#define ST_FAULT_ALLOC 1
#define ST_FAULT_COPY 2
st_status st_inject_fault(int site, int nth);

/* Message for the last non-OK status on this thread. */
const char* st_last_error(void);

#ifdef __cplusplus
}
#endif
#endif

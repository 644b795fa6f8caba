/*
 * FP64 CPU oracle for the differentiable path trace (test infrastructure).
 *
 * This is test infrastructure: only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load it. It shares no code with the CUDA
 * library. Everything is computed in double precision with brute-force
 * (all-triangle) ray intersection.
 *
 * What it computes (the paper's renderer R(x, m, c), Sec. 3.2 "Vertex
 * optimization" and Sec. 3.3 "Material Optimization"):
 *   - the Monte Carlo pixel estimate of a triangle mesh with per-face
 *     Torrance-Sparrow reflectance (Sec. 3.3 "Representation", mesh colors at
 *     resolution r = 0) under point lights and/or an equirectangular HDR
 *     environment (Sec. 3.1), with global illumination (Sec. 3.3 "Effects of
 *     Global Illumination");
 *   - the gradient of sum_p <dL/dI_p, I_p> with respect to vertex positions and
 *     per-face parameters (the quantity an MSE loss as in Sec. 3.2 needs),
 *     interior part by sparse forward-mode dual numbers, primary-visibility
 *     edge part by edge sampling in screen space, secondary-visibility edge
 *     part by edge sampling on each path vertex's sphere of directions.
 * The exact estimator (random-number layout, conventions) is stated in
 * oracle.cpp's header comment.
 */
#ifndef ST_ORACLE_H
#define ST_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int n_vertices, n_faces;
  const double* vertices;    /* [V][3] */
  const int* faces;          /* [F][3] */
  const double* face_params; /* [texels][param_width]: kd_r kd_g kd_b ks (or ks_r ks_g ks_b) roughness */
  int brdf;                  /* 0 = GGX, 1 = Beckmann */
  int n_lights;
  const double* light_pos;   /* [L][3] */
  const double* light_intensity; /* [L][3] radiant intensity, RGB */
  int env_width, env_height; /* 0 if no environment */
  const float* env_rgb;      /* [H][W][3] */
  int color_res;             /* mesh-colors resolution r >= 0; face_params then holds
                                F*(r+1)(r+2)/2 texels of 5 params, texel k(r, t, alpha, beta) */
  int param_width;           /* parameters per texel: 5 (kd rgb, ks, roughness) or 7 (kd rgb, ks rgb,
                                roughness); gradients use the same layout */
  int smooth_normals;        /* 0: flat face normals; 1: shading normals interpolated from vertex normals
                                (each the normalised sum of its faces' e1 x e2), oracle.cpp states the rules */
  int fresnel;               /* 0: Fresnel factor held at ks; 1: Schlick's approximation with F0 = ks */
} orc_scene;

typedef struct {
  float eye[3], target[3], up[3];
  float fov_y_deg;
  int width, height, spp;
  long long pixel_offset;
  int n_lights;                  /* point lights of this view only (0..2), after the scene's */
  float light_pos[2][3];
  float light_intensity[2][3];
} orc_view;

typedef struct {
  int max_bounces;
  unsigned long long seed;
  int edge_mode;    /* 0 = silhouette edges, 1 = every mesh edge */
  int edge_spp;     /* edge samples per pixel; 0 = the view's spp */
  int n_threads;    /* 0 = all hardware threads */
  int secondary;    /* gradients: add the secondary-visibility edge term at every path vertex: 0 = off,
                       1 = one edge picked uniformly, 2 = picked through the edge hierarchy (importance) */
} orc_params;

/* Pixel values for a list of pixels (view index, x, y): out [n][3]. Returns the
 * number of ray queries (segments) traced, or -1 on invalid input. */
long long orc_render_pixels(const orc_scene* s, const orc_view* views, int n_views,
                            const orc_params* p, const int* pix /*[n][3]*/, int n,
                            double* out /*[n][3]*/);

/* Path signatures of the listed pixels: out [n] = the sum over the pixel's
 * samples (mod 2^64) of a 64-bit FNV-1a hash of each path's discrete decisions
 * (faces hit, environment texels drawn, BSDF lobes, shadow-ray visibility; the
 * order is stated in oracle.cpp). Returns segments or -1. */
long long orc_render_signatures(const orc_scene* s, const orc_view* views, int n_views,
                                const orc_params* p, const int* pix, int n, uint64_t* out);

/* Interior gradient for the listed pixels with weights dLdI [n][3] (plus the
 * secondary-visibility edge term at every path vertex when p->secondary):
 * d_verts [V][3] and d_face [texels][5] are ACCUMULATED (+=). Returns segments or -1. */
long long orc_grad_pixels(const orc_scene* s, const orc_view* views, int n_views,
                          const orc_params* p, const int* pix, int n, const double* dLdI,
                          double* d_verts, double* d_face);

/* Primary-visibility edge term over all views; dLdI is the full packed image
 * [sum H*W][3]. Samples whose pixel weight is zero in every channel are not
 * traced (their contribution is exactly zero). d_verts accumulated (+=).
 * Returns segments traced or -1. */
long long orc_edge_grad(const orc_scene* s, const orc_view* views, int n_views,
                        const orc_params* p, const double* dLdI, double* d_verts);

/* Shadow-edge term of point lights on surfaces the camera sees (the boundary
 * term of the image integral across shadow edges; oracle.cpp states the
 * estimator); dLdI is the full packed image. d_verts accumulated (+=).
 * Returns segments traced or -1. */
long long orc_shadow_edge_grad(const orc_scene* s, const orc_view* views, int n_views,
                               const orc_params* p, const double* dLdI, double* d_verts);

/* Number of edge candidates of view v and the per-view sample count. */
int orc_edge_candidates(const orc_scene* s, const orc_view* view, const orc_params* p,
                        int* out_edges /* may be NULL; [2*E] vertex pairs */);

/* One path started at continuous pixel coordinate (px, py) of `view` with
 * counter words (c0, c1, stream); rgb out. If grad_w != NULL the interior
 * gradient of <grad_w, L> is accumulated into d_verts/d_face. Returns segments. */
long long orc_trace_screen(const orc_scene* s, const orc_view* view, const orc_params* p,
                           double px, double py, uint32_t c0, uint32_t c1, uint32_t stream,
                           double* rgb, const double* grad_w, double* d_verts, double* d_face);

/* As orc_trace_screen without gradient, recording (mode 1) or replaying
 * (mode 2) the quantities the gradient holds constant: sampled directions,
 * pdfs, MIS weights and the sampled texel. *tape_len is the capacity on input
 * and the recorded length on output (mode 1). Returns segments, -2 if a replay
 * went out of step, -3 if the tape buffer is too small. */
long long orc_trace_screen_taped(const orc_scene* s, const orc_view* view, const orc_params* p,
                                 double px, double py, uint32_t c0, uint32_t c1, uint32_t stream,
                                 int mode, double* tape, int* tape_len, double* rgb);

/* Microfacet terms D(cos theta_h) and Smith G1(cos theta) at roughness alpha. */
void orc_microfacet(int brdf, double alpha, double c, double* D, double* G1);

/* Brute-force closest hit: rays [n][7] = o, d, tmax; out tri id (-1 miss), t. */
void orc_closest_hit(const orc_scene* s, const double* rays, int n, int exclude_tri,
                     int* out_tri, double* out_t);

/* BRDF value (RGB) times nothing: f(wi, wo) for normal n; out [3]. fresnel as in orc_scene. */
void orc_brdf_eval(int brdf, int fresnel, const double* params5, const double* n, const double* wi,
                   const double* wo, double* out);
/* Mixture sampling pdf (solid angle) of direction wi. */
double orc_brdf_pdf(int brdf, const double* params5, const double* n, const double* wi,
                    const double* wo);
/* Sample a direction from uniforms (ul, u1, u2); returns pdf (0 = invalid). */
double orc_brdf_sample(int brdf, const double* params5, const double* n, const double* wo,
                       double ul, double u1, double u2, double* wi);

/* Philox4x32-10 block: ctr[4], key[2] -> out[4]. */
void orc_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out);

/* Environment alias table: prob[N], alias[N], pmf[N]. Returns 0 on success. */
int orc_env_alias(const float* rgb, int w, int h, double* prob, int* alias, double* pmf);
/* Sample a texel index from raw 32-bit words (u0, u1) with the table. */
int orc_alias_pick(const double* prob, const int* alias, int n, uint32_t u0, uint32_t u1);

/* Mesh-colors texel index k(r, t, alpha, beta) (Sec. 3.3). */
long long orc_mesh_color_index(int r, long long t, double alpha, double beta);

/* Secondary edge pick through the edge hierarchy, for tests: the probability of
 * every edge (pmf [E], edge order) at a vertex p with tangent-plane normal n and
 * band bnd, for silhouette (edge_mode 0) or all-edge sampling; returns E or -1. */
int orc_sec_edge_pmf(const orc_scene* s, const double* p, const double* n, double bnd, int edge_mode, double* pmf);
/* count picks at the same vertex, pick i with the counters (i, c1) of vertex b
 * and stream: edge [count] (-1 if every node is below the plane) and prob. */
int orc_sec_edge_picks(const orc_scene* s, unsigned long long seed, uint32_t c1, int b, uint32_t stream,
                       const double* p, const double* n, double bnd, int edge_mode, const uint32_t* uleaf, int count,
                       int* edge, double* prob);

#ifdef __cplusplus
}
#endif
#endif

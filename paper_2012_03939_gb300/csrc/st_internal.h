// Library-internal scene state shared by the translation units of libst.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "st.h"
#include "st_device.cuh"

namespace st {

// Mesh facts the primary-visibility bins use to drop back faces: six times the
// signed volume (its sign tells outward from inward winding) and the vertex
// bounds as order-preserving ints.
struct MeshStat {
  double vol6;
  int lo[3], hi[3];
  int winding;   // +1 outward, -1 inward, 0 when the volume is too small against the bounds to tell
};

// Per-call arguments the kernels read from device memory, so a captured CUDA
// graph can be replayed with a new seed, new output pointers and new camera
// poses without recapture.
struct CallArgs {
  uint32_t k0, k1;          // Philox key = seed
  float* image;             // forward output
  const float* dLdI;        // backward input
  float* dV;                // backward outputs (accumulated)
  float* dF;
  unsigned long long* sig;  // forward, optional: per-pixel path signatures (image rows)
};

// A contiguous range of the call's job space: camera samples of one view, or
// edge-sample sides of one view.
struct Seg {
  long long base, count;
  int view;
  unsigned kind : 4;        // 0 = camera paths, 1 = edge sides, 2 = shadow-edge sides (two jobs per sample)
  unsigned light : 4;       // kind 2: the view's point light
  unsigned pair : 24;       // kind 2: its (view, light) candidate list
  long long n_samples;      // kinds 1, 2: samples; kind 0: W*H*spp
};
// 32 bytes: every job's lookup reads it (at 40 bytes k_raygen ran a third slower)
static_assert(sizeof(Seg) == 32, "Seg layout");

// Device pointers of the wavefront engine (one chunk of Q path slots).
struct Engine {
  int Q = 0, B = 0, NS = 0;   // capacity, bounces the records were sized for, shadow rays per path
  bool records = false;
  float4 *o = nullptr, *d = nullptr, *thr = nullptr, *rad = nullptr;
  int4* ctr = nullptr;        // Philox counter words (c0, c1, stream) and the vertex index of the first ray
  int2* hit = nullptr;        // (face, t bits)
  int* origin = nullptr;
  int *q0 = nullptr, *q1 = nullptr, *qs = nullptr;
  float4 *sh_dir = nullptr, *sh_c = nullptr;  // [NS][Q]
  float4 *r0 = nullptr, *r1 = nullptr, *r2 = nullptr, *r3 = nullptr;  // [B+1][Q] records
  float4* esc = nullptr;      // escape radiance (rgb, flag)
  int* nb = nullptr;          // hits per path
  unsigned long long* sig = nullptr;  // per-slot path signature (forward calls that ask for them)
  // secondary-visibility edge samples (backward calls that ask for them)
  long long sec_cap = 0;      // job capacity = B * Q (one sample per path vertex)
  float4* sj = nullptr;       // [4][sec_cap]: (p, face), (w, weight), (m, tau), (dL/dI * T, edge)
  int4* sje = nullptr;        // [sec_cap]: (camera counter c0, sample, camera slot, vertex)
  float4* pinj = nullptr;     // [B][Q]: adjoint of each vertex position from its edge sample
  float4* shr = nullptr;      // [3][Q] shadow-edge samples, at the slot of their minus side:
                              // (S, n_S), (q, receiver face), (tau, edge, weight factor, s); S.x NaN = none
  bool shadow = false;
  int* cnt = nullptr;         // counters, see CNT_*
  unsigned long long* stat = nullptr;  // per-call 64-bit statistics, see STAT_*
  long long bytes = 0;
};

// Wavefront engines (buffer sets) of a batched call: consecutive chunks rotate over them, each on its own stream,
// so one chunk's sparse last bounces overlap the next chunks' stages.
constexpr int OVERLAP_ENGINES = 2;

enum { CNT_EXT = 0, CNT_EXT_FETCH = 16, CNT_SHADE_FETCH = 32, CNT_SH = 48, CNT_SH_FETCH = 64, CNT_MISC = 80,
       CNT_SEC = CNT_MISC, CNT_FB = 88, CNT_FB_FETCH = 89, CNT_SIZE = 96 };
enum { STAT_PATHS = 0, STAT_EXT = 1, STAT_SHADOW = 2, STAT_EDGE = 3, STAT_VISITS = 4, STAT_TESTS = 5,
       STAT_SEC = 6, STAT_SH_VISITS = 7, STAT_SH_TESTS = 8, STAT_SIZE = 10 };

struct GraphEntry {
  std::vector<long long> key;
  cudaGraphExec_t exec = nullptr;
  int launches = 0;
};

}  // namespace st

struct st_scene {
  int device = 0;
  int nv = 0, nf = 0, brdf = 0, nl = 0;
  int res = 0, ntex = 1;         // mesh-colors resolution and texels per face
  int builder = 0;               // ST_BVH_PLOC or ST_BVH_LBVH
  int np = 5;                    // caller parameters per texel: 5 (scalar specular) or 7 (RGB specular)
  bool closed = false;           // one surface; every edge has two faces that traverse it in opposite directions
  st::MeshStat* mstat = nullptr; // signed volume and vertex bounds, recomputed on the device after each update
  bool smooth = false;           // interpolated shading normals
  int fresnel = 0;               // ST_FRESNEL_HELD or ST_FRESNEL_SCHLICK
  float4* vnrm = nullptr;        // [V] vertex normal N_v and |M_v| (smooth), recomputed with mstat
  int* vf_start = nullptr;       // [V + 1] faces around each vertex (CSR, face order)
  int* vf_list = nullptr;        // [3F]
  float* dN = nullptr;           // [V][3] backward scratch: adjoint of the vertex normals (smooth)
  // hierarchy over the edges for the secondary pick: blocks of et_G edges, 2^et_L leaves
  int et_G = 4, et_L = 0, et_nleaf = 0;
  float4* et_lo = nullptr;       // [2^(L+1)] box low corner, summed edge length (heap order, root 1)
  float4* et_hi = nullptr;       // [2^(L+1)] box high corner
  float4* et_cn = nullptr;       // [2^(L+1)] cone of the faces' unit normals: axis, cos half-angle (-2: none)
  float* verts = nullptr;        // [V*3]
  int* faces = nullptr;          // [F*3]
  float4* params = nullptr;      // [F*ntex*2] per texel: (kd_r, kd_g, kd_b, ks_r), (roughness, ks_g, ks_b, 0)
  // LBVH
  float4* tri = nullptr;         // [F*3] triangles in leaf order; tri[3i].w = face id bits
  float4* nodes = nullptr;       // [(F-1)*4]
  int* parent = nullptr;         // [F-1] internal parents, then [F] leaf parents
  int* flags = nullptr;          // [F-1] bottom-up visit counters
  uint32_t *keys = nullptr, *keys2 = nullptr;
  int *ids = nullptr, *ids2 = nullptr;
  uint32_t* hist = nullptr;
  int* bounds = nullptr;         // [6] ordered-int centroid bounds
  int sort_blocks = 0;
  // 4-wide BVH collapsed from the binary tree (what the traversal walks)
  float4* nodes4 = nullptr;      // [n4*7]: lo.x[4], hi.x[4], lo.y[4], hi.y[4], lo.z[4], hi.z[4], children[4]
  int* src4 = nullptr;           // [n4*4]: binary node (>= 0) or ~leaf (< 0) behind each child slot
  int* q4 = nullptr;             // [4*F] collapse work queues
  int* c4 = nullptr;             // [2] collapse counters
  int n4 = 0;
  // lights
  float4* lights = nullptr;      // [nl*2]: (pos, 0), (intensity, 0)
  std::vector<st_point_light> host_lights;
  // environment
  st::DevEnv env{};
  float4* env_tex = nullptr;
  float2* env_alias = nullptr;
  // edges (sorted by (min vertex, max vertex))
  int n_edges = 0;
  int2* edge_v = nullptr;
  int2* edge_f = nullptr;        // second face -1 on a boundary; -2 if more than two faces
  int* edge_flag = nullptr;      // [views * E]
  int* edge_cand = nullptr;      // [views * E]
  int* edge_ncand = nullptr;     // [views]
  int edge_cap_views = 0;
  int* sh_flag = nullptr;        // [pairs * E] light-silhouette flags per (view, light)
  int* sh_cand = nullptr;        // [pairs * E] their ordered compaction
  int* sh_ncand = nullptr;       // [pairs]
  int2* d_pairs = nullptr;       // [pairs] (view, light)
  int sh_cap_pairs = 0;
  // primary-visibility bins: per view pixel, the leaves whose screen box covers it
  int* bin_start = nullptr;      // [P + 1] exclusive prefix of the counts
  int* bin_cur = nullptr;        // [P] counts, then fill cursors
  int* bin_list = nullptr;       // [bin_cap] leaf indices
  int* bin_ok = nullptr;         // [views] 1 = the view's primary rays may use the bins
  int* bin_part = nullptr;       // scan block sums
  long long bin_pix_cap = 0;     // cell capacity (bin_start, bin_cur)
  long long bin_cap = 0;         // list capacity
  int bin_views_cap = 0;
  int* bin_total_host = nullptr; // pinned: list length the last call needed
  // the lists are a function of the vertices and of each view's camera, size and cell layout: a call whose key
  // equals the last build's, with no vertex update since, uses them as they are
  bool bins_valid = false;
  unsigned long long bins_geom = 0;     // geom_version of the last build
  std::vector<uint32_t> bins_key;       // views of the last build (bins_key())
  unsigned long long geom_version = 0;  // bumped by every vertex update (refit, rebuild)
  // point-light shadow lists: per scene light an lbin_res x lbin_res frustum of cells (k_light_views), built
  // like the primary-visibility bins; they depend on the vertices only (the scene's lights are fixed)
  st::DevView* d_lviews = nullptr;  // [nl]
  int* lbin_start = nullptr;        // [cells + 1]
  int* lbin_cur = nullptr;          // [cells]
  int* lbin_list = nullptr;         // [lbin_cap]
  int* lbin_ok = nullptr;           // [nl]
  int* lbin_part = nullptr;         // scan block sums
  int* lbin_total_host = nullptr;   // pinned: list length the last build needed
  long long lbin_cells = 0, lbin_cap = 0;
  int lbin_res = 0;
  bool lbins_valid = false;
  unsigned long long lbins_geom = 0;
  float* acc = nullptr;          // [6 * pixels] forward accumulation, compensated FP32 (sum, error) per channel
  unsigned long long* sacc = nullptr;  // [pixels] path-signature sums (bin-space pixel index)
  long long acc_cap = 0;
  // per-call tables
  st::DevView* d_views = nullptr;
  st::Seg* d_segs = nullptr;
  st::CallArgs* d_args = nullptr;
  int view_cap = 0;
  st::Engine eng;
  st::Engine eng2[st::OVERLAP_ENGINES - 1];   // further engines: consecutive chunks of a batched call rotate over all
  cudaStream_t aux_stream[st::OVERLAP_ENGINES - 1] = {};   // their streams (join a captured graph through events)
  std::vector<cudaEvent_t> xev;  // fork, per-chunk resolve and join events of overlapped calls
  int xev_used = 0;
  int* d_err = nullptr;
  // graph cache
  cudaStream_t cap_stream = nullptr;
  std::vector<st::GraphEntry> graphs;
  // timing (time_kernels): event pairs around k_extend launches (0), k_shadow launches (1), and the GPU-side
  // intervals between the host synchronisations of a per-view call (2)
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[3];
  int ev_used[3] = {0, 0, 0};
  int host_syncs = 0;
  int sm_count = 0;
  int g_ext = 0, g_ext_s = 0, g_shade = 0, g_shadow = 0, g_shadow_s = 0;  // stage grids
  long long last_edge_samples = 0;
  int launches = 0;              // kernels enqueued by the last call
  st_stats last{};
};

namespace st {
cudaError_t bvh_build(st_scene* s, cudaStream_t stream);    // Morton order + radix-tree hierarchy + boxes
cudaError_t mesh_stat(st_scene* s, cudaStream_t stream);   // MeshStat (and vertex normals) of the current vertices (no sync)
cudaError_t bvh_build_ploc(st_scene* s, cudaStream_t stream);  // Morton order + PLOC clustering + boxes (synchronises)
cudaError_t bvh_refit(st_scene* s, cudaStream_t stream);    // leaf records + boxes, same order (+ 4-wide boxes)
cudaError_t bvh_collapse(st_scene* s, cudaStream_t stream); // 4-wide tree from the binary one (synchronises)
cudaError_t trace_closest(st_scene* s, const float* rays, int n, int exclude, int* out_tri, float* out_t,
                          cudaStream_t stream);
void set_error(const std::string& msg);
bool fault_now(int site);   // host-side fault injection: true when this event at `site` is to fail
int sort_blocks_for(int n);
}  // namespace st

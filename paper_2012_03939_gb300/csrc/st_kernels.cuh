// Wavefront kernels of the forward path trace, its adjoint and the edge term.
//
// One chunk of Q path slots is processed stage by stage: raygen fills the
// extension queue, then for each bounce b: extend (closest hit), shade
// (flat-normal Torrance-Sparrow vertex: next-event rays to every point light
// and one alias-sampled environment direction, then a BSDF-sampled
// continuation appended to the next queue), shadow (any hit for the NEE rays).
// Queues are compacted with warp-aggregated atomics. Stage kernels are
// persistent: each warp fetches 32 queue entries at a time from a device
// counter, so the same launch works for any queue length (needed for CUDA
// graph replay, where the host never reads the counts).
#pragma once
#include "st_internal.h"
#include "st_trace.cuh"

namespace st {

constexpr unsigned FULL = 0xffffffffu;
constexpr int EXT_BLOCK = 128;
constexpr int ENV_VALID = 1 << 30;
constexpr int ENV_VIS = 1 << 8;

struct KCtx {
  const float* V;
  const int* F;
  const float4* P;
  const float4* nodes;
  const float4* tri;
  int nf, nv;
  int n4;                 // nodes of the 4-wide tree
  const float4* lights;
  int nl, nlt, NS;        // scene lights, + the most any view of the call adds, + environment
  DevEnv env;
  int brdf;
  int fresnel;            // 1: Schlick's Fresnel factor (F0 = ks); 0: held at ks
  int res, ntex;          // mesh-colors resolution r and texels per face
  int np;                 // parameters per texel in the caller's layout: 5 (scalar ks) or 7 (RGB ks)
  const int2* edge_v;
  const int2* edge_f;
  int n_edges;
  int edge_mode;
  int* edge_flag;
  int* edge_cand;
  int* edge_ncand;
  const int* sh_cand;     // shadow edges: candidate lists per (view, light) pair
  const int* sh_ncand;
  const int* bin_start;   // primary-visibility bins (see k_bin)
  const int* bin_list;    // leaf indices per pixel
  int* bin_cur;
  const int* bin_ok;
  long long bin_cap;
  long long bin_pixels;   // pixels of the call (accumulation space)
  long long bin_cells;    // cells of the primary-visibility bins (kb x kb per pixel of each view)
  // point-light shadow lists: per scene light, a frustum from the light around the mesh (k_light_views) whose
  // cells list the leaves a shadow ray to that light may cross (see light_bin_range)
  const DevView* lviews;
  const int* lbin_start;  // nullptr: shadow rays to scene lights traverse the BVH
  const int* lbin_list;
  const int* lbin_ok;     // per scene light: 1 = its shadow rays may use the lists
  long long lbin_cap;
  long long lbin_cells;
  float* acc;             // per-pixel compensated sample sums, (sum, error) x 3 (bin-space pixel index)
  int cull;               // the mesh is one closed, consistently wound surface (see MeshStat)
  const MeshStat* mstat;
  int smooth;             // interpolated shading normals from vn
  const float4* vn;       // [V] vertex normal N_v and |M_v|
  float* dN;              // backward with smooth normals: [V][3] adjoint of the vertex normals
  int sec_tree;           // secondary pick through the edge hierarchy (else uniform)
  int et_G, et_L;         // edges per leaf block, tree levels
  const float4* et_lo;    // tree nodes (heap order): box low corner + summed length, high corner,
  const float4* et_hi;    // cone of the faces' unit normals (axis, cos half-angle; -2 = unbounded)
  const float4* et_cn;
  const DevView* views;
  const Seg* segs;
  int n_segs;
  const CallArgs* args;
  int B;
  int sec;                // backward: secondary-visibility edge samples on
  int sig;                // forward: path signatures on
  unsigned long long* sacc;   // per-pixel signature sums (bin-space pixel index)
  Engine e;
  int* err;
};

__device__ __forceinline__ int find_seg(const Seg* segs, int n, long long job) {
  int lo = 0, hi = n - 1, r = -1;
  while (lo <= hi) {
    int mid = (lo + hi) >> 1;
    if (segs[mid].base <= job) { r = mid; lo = mid + 1; } else hi = mid - 1;
  }
  return r;
}

// all 32 lanes must call; returns this lane's slot in the queue (or -1)
__device__ __forceinline__ int warp_append(int* counter, bool pred) {
  unsigned m = __ballot_sync(FULL, pred);
  int lane = threadIdx.x & 31;
  int base = 0;
  if (m) {
    int leader = __ffs(m) - 1;
    if (lane == leader) base = atomicAdd(counter, __popc(m));
    base = __shfl_sync(FULL, base, leader);
  }
  return pred ? base + __popc(m & ((1u << lane) - 1u)) : -1;
}

// path signatures: FNV-1a step over one 32-bit decision
constexpr unsigned long long SIG_BASIS = 0xcbf29ce484222325ull;
__device__ __forceinline__ void sig_mix(unsigned long long& h, uint32_t x) {
  h = (h ^ (unsigned long long)x) * 0x100000001b3ull;
}

__device__ __forceinline__ float3 fetch_vertex(const float* V, int v) { return mk3(V[3 * v], V[3 * v + 1], V[3 * v + 2]); }

__device__ __forceinline__ Mat fetch_mat(const float4* P, int f) {
  float4 a = __ldg(&P[2 * f]), b = __ldg(&P[2 * f + 1]);   // (kd rgb, ks_r), (roughness, ks_g, ks_b, -)
  Mat m;
  m.kd[0] = a.x; m.kd[1] = a.y; m.kd[2] = a.z;
  m.ks[0] = a.w; m.ks[1] = b.y; m.ks[2] = b.z;
  m.alpha = b.x;
  return m;
}

// Point light j of a path of view vi: the scene's lights, then the view's own.
__device__ __forceinline__ void point_light(const KCtx& c, int vi, int j, float4& lp, float4& li) {
  if (j < c.nl) {
    lp = __ldg(&c.lights[2 * j]);
    li = __ldg(&c.lights[2 * j + 1]);
  } else {
    lp = c.views[vi].vl[2 * (j - c.nl)];
    li = c.views[vi].vl[2 * (j - c.nl) + 1];
  }
}

__device__ __forceinline__ int lights_of(const KCtx& c, int vi) {
  return c.nlt > c.nl ? c.nl + c.views[vi].nvl : c.nl;
}

// Mesh-colors texel of a hit at p on face f (Sec. 3.3): k = (f (r+1)(r+2) +
// i (2r - i + 3)) / 2 + j with (i, j) = floor(r (alpha, beta)), alpha and beta
// the barycentric weights of the face's second and third vertices.
__device__ __forceinline__ int texel_of(const KCtx& c, int f, float3 p, float3 v0, float3 v1, float3 v2) {
  if (c.res == 0) return f;
  float3 e1 = v1 - v0, e2 = v2 - v0, q = p - v0;
  float3 m = cross3(e1, e2);
  float im = 1.0f / dot3(m, m);
  float alpha = dot3(cross3(q, e2), m) * im, beta = dot3(cross3(e1, q), m) * im;
  int r = c.res;
  int i = min(max((int)floorf((float)r * alpha), 0), r);
  int j = min(max((int)floorf((float)r * beta), 0), r - i);
  return f * c.ntex + (i * (2 * r - i + 3)) / 2 + j;
}

// Interpolated shading normal at p on face f (vertices v0, v1, v2): barycentric
// weights b1 = ((p - v0) x e2).m / m.m, b2 = (e1 x (p - v0)).m / m.m, n_s =
// normalise((1 - b1 - b2) N0 + b1 N1 + b2 N2), times sgn (the face normal's turn
// toward the incoming ray).
__device__ __forceinline__ float3 shading_normal(const KCtx& c, int f, float3 p, float3 v0, float3 v1, float3 v2,
                                                 float sgn) {
  float3 e1 = v1 - v0, e2 = v2 - v0, q = p - v0;
  float3 m = cross3(e1, e2);
  float mm = dot3(m, m);
  float b1 = dot3(cross3(q, e2), m) / mm, b2 = dot3(cross3(e1, q), m) / mm;
  float3 n0 = xyz(c.vn[c.F[3 * f]]), n1 = xyz(c.vn[c.F[3 * f + 1]]), n2 = xyz(c.vn[c.F[3 * f + 2]]);
  return norm3(n0 * (1.0f - b1 - b2) + n1 * b1 + n2 * b2) * sgn;
}

// ------------------------------------------------------------------ edges
__device__ __forceinline__ bool facing(const KCtx& c, int f, float3 eye) {
  int a = c.F[3 * f], b = c.F[3 * f + 1], d = c.F[3 * f + 2];
  float3 p0 = fetch_vertex(c.V, a);
  float3 m = cross3(fetch_vertex(c.V, b) - p0, fetch_vertex(c.V, d) - p0);
  return dot3(m, eye - p0) > 0.0f;
}

// screen segment of edge e clipped to the image; false if not drawable
__device__ __forceinline__ bool edge_screen(const KCtx& c, const DevView& v, int e, float2& sa, float2& sb, float& t0,
                                            float& t1) {
  int2 ev = c.edge_v[e];
  if (!cam_project(v, fetch_vertex(c.V, ev.x), sa.x, sa.y)) return false;
  if (!cam_project(v, fetch_vertex(c.V, ev.y), sb.x, sb.y)) return false;
  float dx = sb.x - sa.x, dy = sb.y - sa.y;
  float pp[4] = {-dx, dx, -dy, dy};
  float qq[4] = {sa.x, (float)v.W - sa.x, sa.y, (float)v.H - sa.y};
  t0 = 0.0f; t1 = 1.0f;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (pp[k] == 0.0f) { if (qq[k] < 0.0f) return false; continue; }
    float r = qq[k] / pp[k];
    if (pp[k] < 0.0f) t0 = fmaxf(t0, r); else t1 = fminf(t1, r);
  }
  if (!(t1 > t0)) return false;
  return sqrtf(dx * dx + dy * dy) * (t1 - t0) > 0.0f;
}

__device__ __forceinline__ bool edge_candidate(const KCtx& c, const DevView& v, int e) {
  if (c.edge_mode == 0) {
    int2 ef = c.edge_f[e];
    if (ef.y >= 0 && facing(c, ef.x, v.eye) == facing(c, ef.y, v.eye)) return false;
  }
  float2 sa, sb;
  float t0, t1;
  return edge_screen(c, v, e, sa, sb, t0, t1);
}

struct EdgeSample {
  bool valid;
  int e, px, py;
  float tau, len;
  float2 S, ns;
};

// Sample k of the view's n_samples: candidate t / n_samples for an integer t
// drawn uniformly from [k * nc, (k + 1) * nc) (stratified, probability 1/nc
// per candidate, consecutive samples on the same edge), then a point uniform
// along the candidate's clipped screen segment.
__device__ __forceinline__ EdgeSample edge_sample(const KCtx& c, int vi, const DevView& v, long long k,
                                                  long long n_samples, Key key) {
  EdgeSample s;
  s.valid = false;
  int nc = c.edge_ncand[vi];
  if (nc <= 0) return s;
  U4 u = philox((uint32_t)k, v.off, 0u, 1u, key.k0, key.k1);
  uint64_t t = (uint64_t)k * (uint64_t)nc + (((uint64_t)(u.x >> 8) * (uint64_t)nc) >> 24);
  int i = (int)(t / (uint64_t)n_samples);
  s.e = c.edge_cand[(size_t)vi * c.n_edges + i];
  float2 sa, sb;
  float t0, t1;
  if (!edge_screen(c, v, s.e, sa, sb, t0, t1)) return s;
  s.tau = t0 + unif(u.y) * (t1 - t0);
  float ex = sb.x - sa.x, ey = sb.y - sa.y;
  s.S = make_float2(sa.x + ex * s.tau, sa.y + ey * s.tau);
  s.px = (int)floorf(s.S.x);
  s.py = (int)floorf(s.S.y);
  if (s.px < 0 || s.py < 0 || s.px >= v.W || s.py >= v.H) return s;
  float el = sqrtf(ex * ex + ey * ey);
  s.ns = make_float2(-ey / el, ex / el);
  s.len = el * (t1 - t0);
  s.valid = true;
  return s;
}

__global__ void k_edge_flags(KCtx c, int n_views) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  int vi = blockIdx.y;
  if (e >= c.n_edges || vi >= n_views) return;
  DevView v = c.views[vi];
  c.edge_flag[(size_t)vi * c.n_edges + e] = edge_candidate(c, v, e) ? 1 : 0;
}

// one block per view: ordered compaction of the candidate flags
__global__ void k_edge_compact(KCtx c) {
  __shared__ int part[1024];
  int vi = blockIdx.x;
  const int* fl = c.edge_flag + (size_t)vi * c.n_edges;
  int* out = c.edge_cand + (size_t)vi * c.n_edges;
  int E = c.n_edges;
  int per = (E + 1023) / 1024;
  int b = threadIdx.x * per, en = min(b + per, E);
  int s = 0;
  for (int i = b; i < en; ++i) s += fl[i];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    int v = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  int run = part[threadIdx.x] - s;
  for (int i = b; i < en; ++i)
    if (fl[i]) out[run++] = i;
  if (threadIdx.x == 1023) c.edge_ncand[vi] = part[1023];
}

// ------------------------------------------------------------------ shadow edges (point lights)
// A point light's shadow on a visible surface ends where light rays graze the
// edges that are silhouettes seen from the light. Per (view, light) pair the
// candidates are those edges (or boundary edges) in edge order; sample k picks
// candidate t / N for t uniform in [k n, (k+1) n) and tau uniform on the edge
// (counter (k, pixel_offset, light<<4, 3)); the light ray through y = A +
// tau (B - A), continued from y + SH_EDGE_DELTA |y - L| along it, finds the
// receiver point q = L + s (y - L) on a face other than the edge's own; its
// image S, the screen normal n_S of the
// boundary curve S(tau) (dS/dtau = J_proj(q) s P (B - A), P = I - u n_r^T /
// n_r.u, u = y - L) and |dS/dtau| define the two camera paths at S -+ EDGE_EPS
// n_S. The boundary's screen-normal speed n_S . J_proj(q) dq moves it with the
// edge (dq = s P dy) and with the receiver plane (dq = u ds).
constexpr float SH_EDGE_DELTA = 1e-4f;

__global__ void k_sh_flags(KCtx c, const int2* pairs, int n_pairs, int* flag) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  int pi = blockIdx.y;
  if (e >= c.n_edges || pi >= n_pairs) return;
  int2 pr = pairs[pi];
  float4 lp, li;
  point_light(c, pr.x, pr.y, lp, li);
  int2 ef = c.edge_f[e];
  bool cand = ef.y < 0 || facing(c, ef.x, xyz(lp)) != facing(c, ef.y, xyz(lp));
  flag[(size_t)pi * c.n_edges + e] = cand ? 1 : 0;
}

// Shadow-edge sample of each minus-side slot of the chunk (kind 2), stored at
// that slot for raygen and resolve; S.x = NaN marks no sample.
__global__ void __launch_bounds__(EXT_BLOCK) k_sh_prep(KCtx c, long long j0, int n) {
  __shared__ int sstack[TRACE_SH * EXT_BLOCK];
  const Engine& E = c.e;
  const size_t Q = (size_t)E.Q;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  long long job = j0 + i;
  int si = find_seg(c.segs, c.n_segs, job);
  if (si < 0) return;
  Seg sg = c.segs[si];
  long long local = job - sg.base;
  if (sg.kind != 2 || local >= sg.count || (local & 32)) return;
  const float NaN = __int_as_float(0x7fc00000);
  E.shr[i] = make_float4(NaN, 0, 0, 0);
  long long k = (local >> 6) * 32 + (local & 31);
  if (k >= sg.n_samples) return;
  int nc = c.sh_ncand[sg.pair];
  if (nc <= 0) return;
  DevView v = c.views[sg.view];
  Key key{c.args->k0, c.args->k1};
  U4 u = philox((uint32_t)k, v.off, (uint32_t)sg.light << 4, 3u, key.k0, key.k1);
  uint64_t t = (uint64_t)k * (uint64_t)nc + (((uint64_t)(u.x >> 8) * (uint64_t)nc) >> 24);
  int e = c.sh_cand[(size_t)sg.pair * c.n_edges + (int)(t / (uint64_t)sg.n_samples)];
  float tau = unif(u.y);
  float4 lp, li;
  point_light(c, sg.view, sg.light, lp, li);
  float3 L = xyz(lp);
  int2 ev = c.edge_v[e];
  float3 A = fetch_vertex(c.V, ev.x), Bv = fetch_vertex(c.V, ev.y);
  float3 y = A + (Bv - A) * tau;
  float3 uv = y - L;
  float dy = len3(uv);
  if (!(dy > 0.0f)) return;
  float3 dir = uv * (1.0f / dy);
  float3 org = y + dir * (SH_EDGE_DELTA * dy);
  // the edge's own faces meet that ray only at y: they receive no shadow from it
  int2 ef = c.edge_f[e];
  {
    // the receiver search is a closest-hit query: counted with the extension rays
    unsigned m = __activemask();
    if ((int)(threadIdx.x & 31) == __ffs(m) - 1) atomicAdd(&E.stat[STAT_EXT], (unsigned long long)__popc(m));
  }
  float th;
  int leaf = -1;
  int rf = trace_bvh<false, false, true>(c.nodes, c.tri, c.nf, c.n4, org, dir, __int_as_float(0x7f800000), ef.x, th,
                                         sstack + threadIdx.x, c.err, nullptr, &leaf, ef.y);
  if (rf < 0) return;
  float3 q = org + dir * th;
  float sx, sy;
  if (!cam_project(v, q, sx, sy)) return;
  if (!(sx >= 0.0f && sy >= 0.0f && sx < (float)v.W && sy < (float)v.H)) return;
  float3 r0 = fetch_vertex(c.V, c.F[3 * rf]), r1 = fetch_vertex(c.V, c.F[3 * rf + 1]),
         r2 = fetch_vertex(c.V, c.F[3 * rf + 2]);
  float3 nr = cross3(r1 - r0, r2 - r0);
  float nu = dot3(nr, uv);
  if (!(fabsf(nu) > 0.0f)) return;
  float sc = len3(q - L) / dy;
  float3 ab = Bv - A;
  float3 dq = (ab - uv * (dot3(nr, ab) / nu)) * sc;
  float tx = dot3(cam_project_jt(v, q, 1.0f, 0.0f), dq), ty = dot3(cam_project_jt(v, q, 0.0f, 1.0f), dq);
  float lt = sqrtf(tx * tx + ty * ty);
  if (!(lt > 0.0f)) return;
  E.shr[i] = make_float4(sx, sy, -ty / lt, tx / lt);
  E.shr[Q + i] = make_float4(q.x, q.y, q.z, __int_as_float(rf));
  E.shr[2 * Q + i] = make_float4(tau, __int_as_float(e), (float)nc * lt / (float)sg.n_samples, sc);
}

// ------------------------------------------------------------------ primary-visibility bins
// Every primary ray leaves the eye, so the triangles it can hit are those whose
// projection covers its screen point. Per view and pixel the bins list the
// leaves whose projection, padded by BIN_PAD pixels (plus a relative rounding
// allowance), may overlap the pixel (screen box, then edge functions at the
// pixel's most-inside corner); a primary ray tests its pixel's list with the same watertight test
// and tie rule as the traversal, which therefore finds the same closest hit.
// A view with a triangle straddling the eye plane (projection undefined) keeps
// the BVH for its primary rays.
constexpr float BIN_PAD = 0.02f;
constexpr int BIN_MAX_BOX = 1 << 16;   // a larger screen box sends its view back to the BVH
constexpr int BIN_ILP = 2;              // list entries a lane tests per step


// Screen-space edge functions of a projected triangle, oriented so the inside
// is >= 0, for a conservative pixel-overlap test.
struct ScreenTri {
  float a[3], b[3], c[3];
  bool degenerate;
};

// bin-cell coordinates of a point at rel = X - eye and depth z along fwd (cells: pixels times v.kb)
__device__ __forceinline__ float2 cell_xy(const DevView& v, float3 rel, float z) {
  const float zz = fmaxf(z, Z_NEAR);
  return make_float2((dot3(rel, v.right) / (zz * v.kx) + 1.0f) * (float)(v.W * v.kb) * 0.5f,
                     (1.0f - dot3(rel, v.up) / (zz * v.ky)) * (float)(v.H * v.kb) * 0.5f);
}

// 0: cannot be hit from the eye or off screen; 1: box in (x0..x1, y0..y1);
// -1: view must use the BVH
// Screen coordinates are in bin cells: pixels times v.kb.
__device__ __forceinline__ int leaf_screen_box(const DevView& v, float4 a, float4 b, float4 c, int& x0, int& y0,
                                               int& x1, int& y1, ScreenTri& et) {
  float3 P[3] = {xyz(a), xyz(b), xyz(c)};
  int front = 0, behind = 0;
  float px[3], py[3];
  const int Wc = v.W * v.kb, Hc = v.H * v.kb;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float3 rel = P[k] - v.eye;
    float z = dot3(rel, v.fwd);
    front += z > Z_NEAR;
    behind += z <= 0.0f;
    float2 q = cell_xy(v, rel, z);
    px[k] = q.x;
    py[k] = q.y;
  }
  if (behind == 3) return 0;
  if (front < 3) return -1;
  float lx = fminf(fminf(px[0], px[1]), px[2]) - BIN_PAD, hx = fmaxf(fmaxf(px[0], px[1]), px[2]) + BIN_PAD;
  float ly = fminf(fminf(py[0], py[1]), py[2]) - BIN_PAD, hy = fmaxf(fmaxf(py[0], py[1]), py[2]) + BIN_PAD;
  if (hx < 0.0f || hy < 0.0f || lx >= (float)Wc || ly >= (float)Hc) return 0;
  x0 = max(0, (int)floorf(lx)); y0 = max(0, (int)floorf(ly));
  x1 = min(Wc - 1, (int)floorf(hx)); y1 = min(Hc - 1, (int)floorf(hy));
  if ((long long)(x1 - x0 + 1) * (y1 - y0 + 1) > BIN_MAX_BOX) return -1;
  float area = (px[1] - px[0]) * (py[2] - py[0]) - (py[1] - py[0]) * (px[2] - px[0]);
  et.degenerate = !(fabsf(area) > 1e-6f);
  float sgn = area > 0.0f ? 1.0f : -1.0f;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    int k1 = k == 2 ? 0 : k + 1;
    // E(x, y) = (x - px_k)(py_k1 - py_k) - (y - py_k)(px_k1 - px_k), sign-normalised
    et.a[k] = -sgn * (py[k1] - py[k]);
    et.b[k] = sgn * (px[k1] - px[k]);
    et.c[k] = -(et.a[k] * px[k] + et.b[k] * py[k]);
  }
  return 1;
}

// can any point of cell (x, y), padded by BIN_PAD, lie inside the triangle?
__device__ __forceinline__ bool pixel_may_overlap(const ScreenTri& et, int x, int y) {
  if (et.degenerate) return true;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float cx = et.a[k] > 0.0f ? (float)(x + 1) : (float)x;   // the pixel corner where E is largest
    float cy = et.b[k] > 0.0f ? (float)(y + 1) : (float)y;
    float e = et.a[k] * cx + et.b[k] * cy + et.c[k];
    float tol = BIN_PAD * (fabsf(et.a[k]) + fabsf(et.b[k])) + 1e-4f * (fabsf(et.a[k] * cx) + fabsf(et.b[k] * cy) +
                                                                      fabsf(et.c[k]));
    if (e < -tol) return false;
  }
  return true;
}

__device__ __forceinline__ float from_ordered(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff); }

// A closed, consistently wound surface seen from an eye outside its bounds is
// first hit on a face wound toward the eye (outward when the signed volume is
// positive, MeshStat::winding); faces clearly wound the other way (beyond a 1e-5
// relative band, so edge-on faces stay) can never be a primary ray's closest hit.
__device__ __forceinline__ bool hidden_back_face(const KCtx& c, const DevView& v, float4 a, float4 b, float4 cc) {
  if (!c.cull || !c.mstat) return false;
  int w = c.mstat->winding;
  if (w == 0) return false;
  float3 lo = mk3(from_ordered(c.mstat->lo[0]), from_ordered(c.mstat->lo[1]), from_ordered(c.mstat->lo[2]));
  float3 hi = mk3(from_ordered(c.mstat->hi[0]), from_ordered(c.mstat->hi[1]), from_ordered(c.mstat->hi[2]));
  float m = 1e-4f * fmaxf(hi.x - lo.x, fmaxf(hi.y - lo.y, hi.z - lo.z)) + 1e-6f;
  bool outside = v.eye.x < lo.x - m || v.eye.x > hi.x + m || v.eye.y < lo.y - m || v.eye.y > hi.y + m ||
                 v.eye.z < lo.z - m || v.eye.z > hi.z + m;
  if (!outside) return false;
  float3 n = cross3(xyz(b) - xyz(a), xyz(cc) - xyz(a));
  float3 e = v.eye - xyz(a);
  float f = dot3(n, e), tol = 1e-5f * len3(n) * len3(e);
  return w > 0 ? f < -tol : f > tol;
}

// fill = 0: count leaves per pixel; fill = 1: write them at start + cursor
template <int FILL>
__global__ void k_bin(KCtx c, int n_views, int* ok) {
  int li = blockIdx.x * blockDim.x + threadIdx.x;
  int vi = blockIdx.y;
  if (li >= c.nf || vi >= n_views) return;
  DevView v = c.views[vi];
  if (v.W <= 0) return;   // a light frustum that does not exist (k_light_views)
  int x0, y0, x1, y1;
  ScreenTri et;
  float4 ta = __ldg(&c.tri[3 * li]), tb = __ldg(&c.tri[3 * li + 1]), tc = __ldg(&c.tri[3 * li + 2]);
  if (hidden_back_face(c, v, ta, tb, tc)) return;
  int r = leaf_screen_box(v, ta, tb, tc, x0, y0, x1, y1, et);
  if (r < 0) { if (!FILL) atomicAnd(&ok[vi], 0); return; }
  if (r == 0) return;
  if (FILL && c.bin_start[c.bin_cells] > c.bin_cap) return;   // overflow: every view uses the BVH
  const long long Wc = (long long)v.W * v.kb;
  for (int y = y0; y <= y1; ++y)
    for (int x = x0; x <= x1; ++x) {
      if (!pixel_may_overlap(et, x, y)) continue;
      long long p = v.bin_cell + (long long)y * Wc + x;
      int k = atomicAdd(&c.bin_cur[p], 1);
      if (FILL) {
        long long at = (long long)c.bin_start[p] + k;
        if (at < c.bin_start[p + 1] && at < c.bin_cap) const_cast<int*>(c.bin_list)[at] = li;
        else atomicOr(c.err, ERR_INDEX);
      }
    }
}

// ------------------------------------------------------------------ point-light shadow lists
// A shadow ray from x to a point light L lies on the line through L and x, so
// every triangle it can cross projects, seen from L, onto x's own projection.
// Each scene light gets a square frustum of R x R cells from L around the
// mesh's bounding sphere (centred on MeshStat's box, radius the farthest
// vertex), binned by k_bin like a camera view: the shadow ray tests the leaves
// of x's cell with the traversal's watertight test and bound, so it finds a
// crossing exactly when the traversal does. A closed, consistently wound
// surface lets k_bin drop the faces wound away from L: a segment that enters
// the solid must leave it through a face wound toward L before reaching L,
// which lies outside. A light inside the sphere (or too close to it) has no
// frustum: W = H = 0, ok = 0, and its shadow rays traverse the BVH.
// One block per light: the block finds the radius, thread 0 writes the view.
constexpr int LVIEW_BLOCK = 256;
__global__ void __launch_bounds__(LVIEW_BLOCK) k_light_views(const float4* lights, const float* V, int nv,
                                                             const MeshStat* m, int R, DevView* lv, int* ok) {
  __shared__ float red[LVIEW_BLOCK];
  const int j = blockIdx.x;
  float3 lo = mk3(from_ordered(m->lo[0]), from_ordered(m->lo[1]), from_ordered(m->lo[2]));
  float3 hi = mk3(from_ordered(m->hi[0]), from_ordered(m->hi[1]), from_ordered(m->hi[2]));
  float3 ctr = (lo + hi) * 0.5f;
  float r2 = 0.0f;
  for (int i = threadIdx.x; i < nv; i += LVIEW_BLOCK) {
    float3 d = mk3(V[3 * i], V[3 * i + 1], V[3 * i + 2]) - ctr;
    r2 = fmaxf(r2, dot3(d, d));
  }
  red[threadIdx.x] = r2;
  __syncthreads();
  for (int h = LVIEW_BLOCK / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + h]);
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  float rad = sqrtf(red[0]) * 1.001f + 1e-6f;
  float3 L = xyz(lights[2 * j]);
  float3 dv = ctr - L;
  float d = len3(dv);
  DevView v;
  v.eye = L;
  v.kb = 1;
  v.spp = 1;
  v.off = 0;
  v.pix_off = 0;
  v.bin_base = 0;
  v.nvl = 0;
  v.bin_cell = (long long)j * R * R;
  for (int k = 0; k < 4; ++k) v.vl[k] = make_float4(0, 0, 0, 0);
  if (!(d > 1.02f * rad + 1e-3f)) {
    v.fwd = v.right = v.up = mk3(0, 0, 0);
    v.kx = v.ky = 1.0f;
    v.W = v.H = 0;
    lv[j] = v;
    ok[j] = 0;
    return;
  }
  float3 f = dv * (1.0f / d);
  float3 a = fabsf(f.y) < 0.9f ? mk3(0, 1, 0) : mk3(1, 0, 0);
  float3 r = norm3(cross3(f, a));
  v.fwd = f;
  v.right = r;
  v.up = cross3(r, f);
  float sn = rad / d;
  v.kx = v.ky = 1.01f * sn / sqrtf(1.0f - sn * sn);   // tangent of the sphere's half-angle, with a margin
  v.W = v.H = R;
  lv[j] = v;
}

// the list of shadow rays from p to scene light j, or (-1, -1): traverse the BVH
__device__ __forceinline__ int2 light_bin_range(const KCtx& c, int j, float3 p) {
  if (c.lbin_start == nullptr || !c.lbin_ok[j] || c.lbin_start[c.lbin_cells] > c.lbin_cap) return make_int2(-1, -1);
  const DevView& v = c.lviews[j];
  float3 rel = p - v.eye;
  float z = dot3(rel, v.fwd);
  if (!(z > Z_NEAR) || v.W <= 0) return make_int2(-1, -1);
  float2 q = cell_xy(v, rel, z);
  int x = (int)floorf(q.x), y = (int)floorf(q.y);
  if (!(q.x >= 0.0f) || !(q.y >= 0.0f) || x >= v.W || y >= v.H) return make_int2(-1, -1);
  long long k = v.bin_cell + (long long)y * v.W + x;
  return make_int2(c.lbin_start[k], c.lbin_start[k + 1]);
}

// any hit of the ray (o, d) before tmax among the listed leaves, skipping face `exclude`: the traversal's leaf
// test, BIN_ILP entries at a time
template <bool STATS>
__device__ __forceinline__ bool bin_any_hit(const KCtx& c, float3 o, float3 d, float tmax, int exclude, int2 br,
                                            TraceStats* ts) {
  RayPre rp = ray_pre(o, d);
  if (br.y > c.lbin_cap || br.x > br.y) { atomicOr(c.err, ERR_INDEX); return false; }
  for (int k = br.x; k < br.y; k += BIN_ILP) {
    int li[BIN_ILP];
    bool bad = false;
#pragma unroll
    for (int u = 0; u < BIN_ILP; ++u) {
      li[u] = k + u < br.y ? __ldg(&c.lbin_list[k + u]) : -1;
      bad |= k + u < br.y && (unsigned)li[u] >= (unsigned)c.nf;
    }
    if (bad) {
      atomicOr(c.err, ERR_INDEX);
      continue;
    }
    float4 ta[BIN_ILP], tb[BIN_ILP], tc[BIN_ILP];
#pragma unroll
    for (int u = 0; u < BIN_ILP; ++u) {
      int l = li[u] >= 0 ? li[u] : li[0];
      ta[u] = __ldg(&c.tri[3 * l]);
      tb[u] = __ldg(&c.tri[3 * l + 1]);
      tc[u] = __ldg(&c.tri[3 * l + 2]);
    }
#pragma unroll
    for (int u = 0; u < BIN_ILP; ++u) {
      if (li[u] < 0) continue;
      if (STATS) ts->tests++;
      if (__float_as_int(ta[u].w) == exclude) continue;
      if (tri_test(rp, xyz(ta[u]), xyz(tb[u]), xyz(tc[u]), tmax) > 0.0f) return true;
    }
  }
  return false;
}

__device__ __forceinline__ int view_of_pixel(const KCtx& c, int n_views, long long p) {
  int lo = 0, hi = n_views - 1, vi = 0;
  while (lo <= hi) {
    int mid = (lo + hi) >> 1;
    if (c.views[mid].bin_base <= p) { vi = mid; lo = mid + 1; } else hi = mid - 1;
  }
  return vi;
}

// forward calls accumulate every pixel's samples in double, in sample order, so
// neither the sample count nor the chunking changes the result
__global__ void k_zero_acc(KCtx c) {
  long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= c.bin_pixels) return;
  float2* a = reinterpret_cast<float2*>(c.acc) + 3 * p;
  a[0] = make_float2(0.0f, 0.0f); a[1] = make_float2(0.0f, 0.0f); a[2] = make_float2(0.0f, 0.0f);
  if (c.sig) c.sacc[p] = 0ull;
}

// image rows of every view = mean of the samples (the output pointer comes from
// the per-call arguments, so a captured graph writes wherever the call asks)
__global__ void k_finish_views(KCtx c, int n_views) {
  long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= c.bin_pixels) return;
  const DevView& v = c.views[view_of_pixel(c, n_views, p)];
  float* img = c.args->image + 3 * (v.pix_off + (p - v.bin_base));
  const float2* a = reinterpret_cast<const float2*>(c.acc) + 3 * p;
  float inv = 1.0f / (float)v.spp;
  img[0] = (a[0].x - a[0].y) * inv;   // compensated sum: running sum minus the carried error
  img[1] = (a[1].x - a[1].y) * inv;
  img[2] = (a[2].x - a[2].y) * inv;
  if (c.sig && c.args->sig) c.args->sig[v.pix_off + (p - v.bin_base)] = c.sacc[p];
}

__global__ void k_fill_int(int* a, int n, int value) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = value;
}

// exclusive scan of n counts into out[0..n] (out[n] = total): per-block scans,
// one block for the block sums, then the add-back
constexpr int SCAN_BLOCK = 1024, SCAN_ITEMS = 4;
__global__ void k_scan_blocks(const int* in, int* out, long long n, int* part) {
  __shared__ int sh[SCAN_BLOCK];
  long long base = (long long)blockIdx.x * SCAN_BLOCK * SCAN_ITEMS + (long long)threadIdx.x * SCAN_ITEMS;
  int v[SCAN_ITEMS];
  int s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) { v[k] = base + k < n ? in[base + k] : 0; s += v[k]; }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int off = 1; off < SCAN_BLOCK; off <<= 1) {
    int t = threadIdx.x >= off ? sh[threadIdx.x - off] : 0;
    __syncthreads();
    sh[threadIdx.x] += t;
    __syncthreads();
  }
  int run = sh[threadIdx.x] - s;
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
  if (threadIdx.x == SCAN_BLOCK - 1) part[blockIdx.x] = sh[SCAN_BLOCK - 1];
}

__global__ void k_scan_parts(int* part, int nb, int* out, long long n) {
  __shared__ int sh[SCAN_BLOCK];
  int per = (nb + SCAN_BLOCK - 1) / SCAN_BLOCK;
  int b = threadIdx.x * per, e = min(b + per, nb);
  long long s = 0;
  for (int i = b; i < e; ++i) s += part[i];
  sh[threadIdx.x] = (int)min(s, (long long)0x7fffffff);
  __syncthreads();
  for (int off = 1; off < SCAN_BLOCK; off <<= 1) {
    int t = threadIdx.x >= off ? sh[threadIdx.x - off] : 0;
    __syncthreads();
    sh[threadIdx.x] = (int)min((long long)sh[threadIdx.x] + t, (long long)0x7fffffff);
    __syncthreads();
  }
  long long run = sh[threadIdx.x] - s;
  for (int i = b; i < e; ++i) { int c2 = part[i]; part[i] = (int)run; run += c2; }
  if (threadIdx.x == SCAN_BLOCK - 1) out[n] = sh[SCAN_BLOCK - 1];
}

__global__ void k_scan_add(int* out, long long n, const int* part) {
  long long i = (long long)blockIdx.x * SCAN_BLOCK * SCAN_ITEMS + threadIdx.x;
  int add = part[blockIdx.x];
#pragma unroll
  for (int k = 0; k < SCAN_ITEMS; ++k, i += SCAN_BLOCK)
    if (i < n) out[i] += add;
}

// the list of bin cell (x, y) of view vi (cells: v.kb x v.kb per pixel)
__device__ __forceinline__ int2 bin_range(const KCtx& c, int vi, const DevView& v, int x, int y) {
  if (c.bin_start == nullptr || !c.bin_ok[vi] || c.bin_start[c.bin_cells] > c.bin_cap) return make_int2(-1, -1);
  if (x < 0 || y < 0 || x >= v.W * v.kb || y >= v.H * v.kb) return make_int2(-1, -1);
  long long p = v.bin_cell + (long long)y * ((long long)v.W * v.kb) + x;
  return make_int2(c.bin_start[p], c.bin_start[p + 1]);
}

// the cell of a camera sample at pixel (x, y) + the 24-bit jitter words ux, uy: exact in integers
__device__ __forceinline__ int2 sample_cell(const DevView& v, int x, int y, uint32_t ux, uint32_t uy) {
  return make_int2(x * v.kb + (int)(((ux >> 8) * (uint32_t)v.kb) >> 24),
                   y * v.kb + (int)(((uy >> 8) * (uint32_t)v.kb) >> 24));
}

// ------------------------------------------------------------------ chunk stages
__global__ void k_reset(int* cnt) {
  for (int i = threadIdx.x; i < CNT_SIZE; i += blockDim.x) cnt[i] = 0;
}

// The closest hit of a first ray from the leaves listed for its bin cell:
// BIN_ILP entries at a time, tested against the same bound and merged in list
// order, which gives what a sequential scan gives (smallest t, ties to the lower
// face id).
template <bool STATS>
__device__ __forceinline__ int2 bin_closest(const KCtx& c, float3 o, float3 d, int2 br, int& tests) {
  RayPre rp = ray_pre(o, d);
  float t = __int_as_float(0x7f800000);
  int f = -1, fl = -1;
  if (br.y > c.bin_cap || br.x > br.y) { atomicOr(c.err, ERR_INDEX); br.y = br.x; }
  for (int k = br.x; k < br.y; k += BIN_ILP) {
    int li[BIN_ILP];
    bool bad = false;
#pragma unroll
    for (int u = 0; u < BIN_ILP; ++u) {
      li[u] = k + u < br.y ? __ldg(&c.bin_list[k + u]) : -1;
      bad |= k + u < br.y && (unsigned)li[u] >= (unsigned)c.nf;
    }
    if (bad) {
      atomicOr(c.err, ERR_INDEX);
      continue;
    }
    float4 ta[BIN_ILP], tb[BIN_ILP], tc[BIN_ILP];
#pragma unroll
    for (int u = 0; u < BIN_ILP; ++u) {
      int l = li[u] >= 0 ? li[u] : li[0];
      ta[u] = __ldg(&c.tri[3 * l]);
      tb[u] = __ldg(&c.tri[3 * l + 1]);
      tc[u] = __ldg(&c.tri[3 * l + 2]);
    }
    float tmax = t * 1.0000001f + 1e-30f;
#pragma unroll
    for (int u = 0; u < BIN_ILP; ++u) {
      float h = li[u] >= 0 ? tri_test(rp, xyz(ta[u]), xyz(tb[u]), xyz(tc[u]), tmax) : -1.0f;
      int fu = __float_as_int(ta[u].w);
      if (h > 0.0f && (h < t || (h == t && fu < f))) { t = h; f = fu; fl = li[u]; }
      if (STATS && li[u] >= 0) tests++;
    }
  }
  return make_int2(fl, __float_as_int(t));
}

// SH: the chunk holds shadow-edge side jobs (kind 2); chunks without them run
// the variant without that branch, whose code is the hot path's. A first ray
// whose view has primary-visibility bins finds its closest hit here, from the
// leaves of its cell (bin_closest); the others are queued (q1, CNT_FB) for
// k_extend's BVH traversal.
template <bool SH, bool STATS>
__global__ void k_raygen(KCtx c, long long j0, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  const Engine& E = c.e;
  bool ok = false, fb = false;
  int tests = 0;
  float3 o = mk3(0, 0, 0), d = mk3(0, 0, 1);
  int4 ct = make_int4(0, 0, 0, 0);
  int2 br = make_int2(-1, -1);
  if (i < n) {
    long long job = j0 + i;
    int si = find_seg(c.segs, c.n_segs, job);
    if (si >= 0) {
      Seg sg = c.segs[si];
      long long local = job - sg.base;
      if (local < sg.count) {
        DevView v = c.views[sg.view];
        Key key{c.args->k0, c.args->k1};
        if (sg.kind == 0) {
          // a segment holds at most 2^31 jobs, so 32-bit division suffices
          unsigned lj = (unsigned)local, pixel = lj / (unsigned)v.spp;
          int s = (int)(lj - pixel * (unsigned)v.spp);
          int x = (int)(pixel % (unsigned)v.W), y = (int)(pixel / (unsigned)v.W);
          uint32_t c0 = v.off + (uint32_t)pixel;
          U4 u = philox(c0, (uint32_t)s, 0u, 0u, key.k0, key.k1);
          d = cam_dir(v, (float)x + unif(u.x), (float)y + unif(u.y));
          o = v.eye;
          ct = make_int4((int)c0, s, 0, sg.view << 4);
          int2 cell = sample_cell(v, x, y, u.x, u.y);
          br = bin_range(c, sg.view, v, cell.x, cell.y);
          ok = true;
        } else if (SH && sg.kind == 2) {
          // shadow-edge sides: the sample is stored at the block's minus slot
          float4 r = E.shr[i - ((local & 32) ? 32 : 0)];
          if (r.x == r.x) {
            float sg2 = (local & 32) ? EDGE_EPS : -EDGE_EPS;
            float sx = r.x + sg2 * r.z, sy = r.y + sg2 * r.w;
            long long k = (local >> 6) * 32 + (local & 31);
            d = cam_dir(v, sx, sy);
            o = v.eye;
            br = bin_range(c, sg.view, v, (int)floorf(sx * (float)v.kb), (int)floorf(sy * (float)v.kb));
            ct = make_int4((int)(uint32_t)k, (int)v.off, 4 + sg.light, sg.view << 4);
            ok = true;
          }
        } else {
          // block of 64 jobs: minus sides of samples 32b..32b+31, then their plus sides
          long long k = (local >> 6) * 32 + (local & 31);
          EdgeSample es;
          es.valid = false;
          if (k < sg.n_samples) es = edge_sample(c, sg.view, v, k, sg.n_samples, key);
          if (es.valid) {
            float sg2 = (local & 32) ? EDGE_EPS : -EDGE_EPS;
            float sx = es.S.x + sg2 * es.ns.x, sy = es.S.y + sg2 * es.ns.y;
            d = cam_dir(v, sx, sy);
            o = v.eye;
            br = bin_range(c, sg.view, v, (int)floorf(sx * (float)v.kb), (int)floorf(sy * (float)v.kb));
            ct = make_int4((int)(uint32_t)k, (int)v.off, 2, sg.view << 4);
            ok = true;
          }
        }
      }
    }
    E.rad[i] = make_float4(0, 0, 0, 0);
    if (E.records) {
      E.nb[i] = 0;
      E.esc[i] = make_float4(0, 0, 0, 0);
      E.r1[i] = make_float4(d.x, d.y, d.z, 0.0f);
    }
    if (ok) {
      if (c.sig) E.sig[i] = SIG_BASIS;
      E.o[i] = make_float4(o.x, o.y, o.z, 0.0f);
      E.d[i] = make_float4(d.x, d.y, d.z, 0.0f);
      E.thr[i] = make_float4(1, 1, 1, 0);
      E.origin[i] = -1;
      E.ctr[i] = ct;
      if (br.x >= 0) E.hit[i] = bin_closest<STATS>(c, o, d, br, tests);
      else fb = true;
    }
  }
  int q = warp_append(&E.cnt[CNT_EXT + 0], ok);
  if (ok) E.q0[q] = i;
  int qf = warp_append(&E.cnt[CNT_FB], fb);
  if (fb) E.q1[qf] = i;
  unsigned m = __ballot_sync(FULL, ok);
  if ((threadIdx.x & 31) == 0 && m) {
    atomicAdd(&E.stat[STAT_PATHS], (unsigned long long)__popc(m));
    atomicAdd(&E.stat[STAT_EXT], (unsigned long long)__popc(m));   // every first ray is a closest-hit query
  }
  if (STATS) {
    for (int off = 16; off > 0; off >>= 1) tests += __shfl_xor_sync(FULL, tests, off);
    if ((threadIdx.x & 31) == 0 && tests) atomicAdd(&E.stat[STAT_TESTS], (unsigned long long)tests);
  }
}

// persistent fetch: a warp takes 32 consecutive queue entries per step
#define ST_WARP_LOOP(total_expr, fetch_ptr)                                      \
  const int lane_ = threadIdx.x & 31;                                          \
  const int total_ = (total_expr);                                             \
  for (;;) {                                                                   \
    int base_ = 0;                                                             \
    if (lane_ == 0) base_ = total_ > 0 ? atomicAdd((fetch_ptr), 32) : 0;       \
    base_ = __shfl_sync(FULL, base_, 0);                                       \
    if (base_ >= total_) break;                                                \
    const int qi_ = base_ + lane_;                                             \
    const bool live_ = qi_ < total_;

#define ST_WARP_LOOP_END }

// Closest hits through the BVH: the rays of bounce b, or with fb = 1 the first
// rays k_raygen queued because no bin cell serves them.
template <bool STATS>
__global__ void __launch_bounds__(EXT_BLOCK) k_extend(KCtx c, int b, int fb) {
  __shared__ int sstack[TRACE_SH * EXT_BLOCK];
  const Engine& E = c.e;
  const int* q = fb ? E.q1 : (b & 1) ? E.q1 : E.q0;
  TraceStats ts{0, 0};
  ST_WARP_LOOP(fb ? E.cnt[CNT_FB] : E.cnt[CNT_EXT + b], fb ? &E.cnt[CNT_FB_FETCH] : &E.cnt[CNT_EXT_FETCH + b])
  if (live_) {
    int slot = q[qi_];
    float4 o = E.o[slot], d = E.d[slot];
    float t = __int_as_float(0x7f800000);
    int fl = -1;
    trace_bvh<false, STATS>(c.nodes, c.tri, c.nf, c.n4, xyz(o), xyz(d), __int_as_float(0x7f800000), E.origin[slot], t,
                            sstack + threadIdx.x, c.err, &ts, &fl);
    E.hit[slot] = make_int2(fl, __float_as_int(t));   // leaf index: shading reads the contiguous leaf record
  }
  ST_WARP_LOOP_END
  if (!fb && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&E.stat[STAT_EXT], (unsigned long long)E.cnt[CNT_EXT + b]);
  if (STATS) {
    for (int off = 16; off > 0; off >>= 1) {
      ts.visits += __shfl_xor_sync(FULL, ts.visits, off);
      ts.tests += __shfl_xor_sync(FULL, ts.tests, off);
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(&E.stat[STAT_VISITS], (unsigned long long)ts.visits);
      atomicAdd(&E.stat[STAT_TESTS], (unsigned long long)ts.tests);
    }
  }
}

__global__ void k_shade(KCtx c, int b) {
  const Engine& E = c.e;
  const int* qin = (b & 1) ? E.q1 : E.q0;
  int* qout = (b & 1) ? E.q0 : E.q1;
  const size_t Q = (size_t)E.Q;
  Key key{c.args->k0, c.args->k1};
  ST_WARP_LOOP(E.cnt[CNT_EXT + b], &E.cnt[CNT_SHADE_FETCH + b])
  bool sh_any = false, cont = false;
  int slot = live_ ? qin[qi_] : 0;
  if (live_) {
    int2 h = E.hit[slot];
    int4 ct = E.ctr[slot];
    const int vb = b + (ct.w & 15);   // path vertex this ray finds (side paths of edge samples start past 0)
    const int vi = ct.w >> 4;         // the path's view (its own lights)
    float4 o4 = E.o[slot], d4 = E.d[slot];
    float3 dir = xyz(d4);
    float3 T = xyz(E.thr[slot]);
    unsigned long long hs = c.sig ? E.sig[slot] : 0ull;
    if (h.x < 0) {
      if (c.sig) { sig_mix(hs, 0xffffffffu); E.sig[slot] = hs; }
      if (c.env.w > 0) {
        float st_;
        int tx = env_texel(c.env, dir, st_);
        if (c.sig) { sig_mix(hs, (uint32_t)tx); E.sig[slot] = hs; }   // the nearest-texel lookup is a decision
        float4 te = __ldg(&c.env.tex[tx]);
        float w = 1.0f;
        if (b > 0) {
          float pe = env_pdf(c.env, te.w, st_);
          float lp = d4.w;
          w = lp * lp / (lp * lp + pe * pe);
        }
        float3 Lw = mk3(te.x, te.y, te.z) * w;
        float4 r = E.rad[slot];
        E.rad[slot] = make_float4(r.x + T.x * Lw.x, r.y + T.y * Lw.y, r.z + T.z * Lw.z, 0.0f);
        if (E.records && b > 0) E.esc[slot] = make_float4(Lw.x, Lw.y, Lw.z, 1.0f);
      }
    } else if (vb < c.B) {        // a ray past the last vertex adds nothing where it hits
      float4 ta = __ldg(&c.tri[3 * h.x]), tb = __ldg(&c.tri[3 * h.x + 1]), tc = __ldg(&c.tri[3 * h.x + 2]);
      int f = __float_as_int(ta.w);
      float t = __int_as_float(h.y);
      float3 p = xyz(o4) + dir * t;
      float3 v0 = xyz(ta), v1 = xyz(tb), v2 = xyz(tc);
      float3 ng = norm3(cross3(v1 - v0, v2 - v0));
      float3 wo = -dir;
      float3 n = dot3(ng, wo) < 0.0f ? -ng : ng;
      // shading normal: n, or interpolated; a direction counts only above both
      float3 ns = c.smooth ? shading_normal(c, f, p, v0, v1, v2, dot3(ng, wo) < 0.0f ? -1.0f : 1.0f) : n;
      int tex = texel_of(c, f, p, v0, v1, v2);
      Mat m = fetch_mat(c.P, tex);
      if (c.sig) sig_mix(hs, (uint32_t)f);
      if (c.sig && c.res > 0) sig_mix(hs, (uint32_t)tex);   // so is the mesh-colors texel
      if (E.records) {
        E.r0[b * Q + slot] = make_float4(p.x, p.y, p.z, __int_as_float(f));
        E.nb[slot] = b + 1;
      }
      const int nlp = lights_of(c, vi);
      for (int j = 0; j < c.nlt; ++j) {
        float4 lp = make_float4(0, 0, 1, 0), li = make_float4(0, 0, 0, 0);
        if (j < nlp) point_light(c, vi, j, lp, li);
        float3 dv = xyz(lp) - p;
        float dist = len3(dv);
        float3 wi = dv * (1.0f / dist);
        float ci = dot3(n, wi);
        bool valid = j < nlp && ci > 0.0f && dist > 2.0f * T_EPS && (!c.smooth || dot3(ns, wi) > 0.0f);
        float3 cc = mk3(0, 0, 0);
        if (valid) cc = mul(mul(T, brdf_cos(c.brdf, c.fresnel, m, ns, wi, wo)), xyz(li)) * (1.0f / (dist * dist));
        E.sh_dir[j * Q + slot] = make_float4(wi.x, wi.y, wi.z, dist - T_EPS);
        E.sh_c[j * Q + slot] = make_float4(cc.x, cc.y, cc.z, valid ? 1.0f : 0.0f);
        sh_any |= valid;
      }
      int flags = 0;
      float3 ewi = mk3(0, 0, 0), escale = mk3(0, 0, 0);
      if (c.env.w > 0) {
        U4 u = philox((uint32_t)ct.x, (uint32_t)ct.y, (uint32_t)(vb << 4) | 1u, (uint32_t)ct.z, key.k0, key.k1);
        int tx = env_pick(c.env, u.x, u.y);
        if (c.sig) sig_mix(hs, (uint32_t)tx);
        int row = tx / c.env.w, col = tx - row * c.env.w;
        float uu = ((float)col + unif(u.z)) / (float)c.env.w, vq = ((float)row + unif(u.w)) / (float)c.env.h;
        float sth, cth, sph, cph;
        sincosf(PI_F * vq, &sth, &cth);
        sincosf(2.0f * PI_F * uu, &sph, &cph);
        ewi = mk3(-sth * sph, cth, sth * cph);
        bool valid = sth > 0.0f && dot3(n, ewi) > 0.0f && (!c.smooth || dot3(ns, ewi) > 0.0f);
        float3 cc = mk3(0, 0, 0);
        if (valid) {
          float4 te = __ldg(&c.env.tex[tx]);
          float pe = env_pdf(c.env, te.w, sth);
          float w = 1.0f;
          if (vb < c.B - 1) {
            float pb = brdf_pdf(c.brdf, m, ns, ewi, wo);
            w = pe * pe / (pe * pe + pb * pb);
          }
          escale = mk3(te.x, te.y, te.z) * (w / pe);
          cc = mul(mul(T, brdf_cos(c.brdf, c.fresnel, m, ns, ewi, wo)), escale);
          flags |= ENV_VALID;
        }
        E.sh_dir[c.nlt * Q + slot] = make_float4(ewi.x, ewi.y, ewi.z, __int_as_float(0x7f800000));
        E.sh_c[c.nlt * Q + slot] = make_float4(cc.x, cc.y, cc.z, valid ? 1.0f : 0.0f);
        sh_any |= valid;
      }
      if (E.records) {
        E.r2[b * Q + slot] = make_float4(ewi.x, ewi.y, ewi.z, __int_as_float(flags));
        E.r3[b * Q + slot] = make_float4(escale.x, escale.y, escale.z, __int_as_float(tex));
      }
      E.o[slot] = make_float4(p.x, p.y, p.z, 0.0f);
      E.origin[slot] = f;          // excluded by this vertex's shadow rays and by its continuation
      if (vb < c.B - 1) {
        U4 u = philox((uint32_t)ct.x, (uint32_t)ct.y, (uint32_t)(vb << 4) | 2u, (uint32_t)ct.z, key.k0, key.k1);
        float3 wi;
        float pdf = brdf_sample(c.brdf, m, ns, wo, unif(u.x), unif(u.y), unif(u.z), wi);
        if (c.smooth && pdf > 0.0f && !(dot3(n, wi) > 0.0f)) pdf = 0.0f;   // below the face
        if (c.sig) sig_mix(hs, (unif(u.x) < lobe_prob(m) ? 1u : 0u) | (pdf > 0.0f ? 2u : 0u));
        if (pdf > 0.0f) {
          float3 Qv = brdf_cos(c.brdf, c.fresnel, m, ns, wi, wo);
          T = mul(T, Qv) * (1.0f / pdf);
          E.thr[slot] = make_float4(T.x, T.y, T.z, 0.0f);
          E.d[slot] = make_float4(wi.x, wi.y, wi.z, pdf);
          if (E.records) E.r1[(b + 1) * Q + slot] = make_float4(wi.x, wi.y, wi.z, pdf);
          cont = true;
        }
      }
      if (c.sig) E.sig[slot] = hs;
    }
  }
  int qs = warp_append(&E.cnt[CNT_SH + b], sh_any);
  if (sh_any) E.qs[qs] = slot;
  int qn = warp_append(&E.cnt[CNT_EXT + b + 1], cont);
  if (cont) qout[qn] = slot;
  ST_WARP_LOOP_END
}

template <bool STATS>
__global__ void __launch_bounds__(EXT_BLOCK) k_shadow(KCtx c, int b) {
  __shared__ int sstack[TRACE_SH * EXT_BLOCK];
  const Engine& E = c.e;
  const size_t Q = (size_t)E.Q;
  int traced = 0;
  TraceStats ts{0, 0};
  ST_WARP_LOOP(E.cnt[CNT_SH + b], &E.cnt[CNT_SH_FETCH + b])
  if (live_) {
    int slot = E.qs[qi_];
    float3 p = xyz(E.o[slot]);
    int exclude = E.origin[slot];
    float3 L = mk3(0, 0, 0);
    int vis = 0;
    for (int k = 0; k < c.NS; ++k) {
      float4 sc = E.sh_c[k * Q + slot];
      if (sc.w == 0.0f) continue;
      float4 sd = E.sh_dir[k * Q + slot];
      float t;
      ++traced;
      int2 lr = k < c.nl ? light_bin_range(c, k, p) : make_int2(-1, -1);
      int hf = lr.x >= 0 ? (bin_any_hit<STATS>(c, p, xyz(sd), sd.w, exclude, lr, &ts) ? 0 : -1)
                         : trace_bvh<true, STATS>(c.nodes, c.tri, c.nf, c.n4, p, xyz(sd), sd.w, exclude, t,
                                                  sstack + threadIdx.x, c.err, &ts);
      if (hf < 0) {
        L += xyz(sc);
        vis |= (k < c.nlt) ? (1 << k) : ENV_VIS;
      }
    }
    float4 r = E.rad[slot];
    E.rad[slot] = make_float4(r.x + L.x, r.y + L.y, r.z + L.z, 0.0f);
    if (c.sig) {
      unsigned long long hs = E.sig[slot];
      sig_mix(hs, (uint32_t)vis);
      E.sig[slot] = hs;
    }
    if (E.records && vis) {
      float4 r2 = E.r2[b * Q + slot];
      E.r2[b * Q + slot] = make_float4(r2.x, r2.y, r2.z, __int_as_float(__float_as_int(r2.w) | vis));
    }
  }
  ST_WARP_LOOP_END
  for (int off = 16; off > 0; off >>= 1) traced += __shfl_xor_sync(FULL, traced, off);
  if ((threadIdx.x & 31) == 0 && traced) atomicAdd(&E.stat[STAT_SHADOW], (unsigned long long)traced);
  if (STATS) {
    for (int off = 16; off > 0; off >>= 1) {
      ts.visits += __shfl_xor_sync(FULL, ts.visits, off);
      ts.tests += __shfl_xor_sync(FULL, ts.tests, off);
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(&E.stat[STAT_SH_VISITS], (unsigned long long)ts.visits);
      atomicAdd(&E.stat[STAT_SH_TESTS], (unsigned long long)ts.tests);
    }
  }
}

// Compensated (Kahan) summation in FP32: (sum, carried error); FP64 adds would
// run on this part's slow FP64 pipe. Same order of operations, same result.
__device__ __forceinline__ void kahan_add(float2& a, float x) {
  float y = __fsub_rn(x, a.y);
  float t = __fadd_rn(a.x, y);
  a.y = __fsub_rn(__fsub_rn(t, a.x), y);
  a.x = t;
}

// the pixel's compensated accumulator takes its samples in sample order, so the
// result does not depend on where chunk boundaries fall. The block stages its
// slots' radiance in shared memory with coalesced loads; the thread holding a
// pixel's first sample then sums that pixel's run in order.
constexpr int RESOLVE_BLOCK = 256;
__global__ void __launch_bounds__(RESOLVE_BLOCK) k_resolve(KCtx c, long long j0, int n) {
  __shared__ float4 srad[RESOLVE_BLOCK];
  const int i0 = blockIdx.x * RESOLVE_BLOCK;
  const int i = i0 + threadIdx.x;
  if (i < n) srad[threadIdx.x] = c.e.rad[i];
  __syncthreads();
  if (i >= n) return;
  long long job = j0 + i;
  int si = find_seg(c.segs, c.n_segs, job);
  if (si < 0) return;
  Seg sg = c.segs[si];
  long long local = job - sg.base;
  if (sg.kind != 0 || local >= sg.count) return;
  DevView v = c.views[sg.view];
  long long pixel = local / v.spp;
  int s = (int)(local - pixel * v.spp);
  if (s != 0 && i != 0) return;
  if (v.bin_base + pixel >= c.bin_pixels) { atomicOr(c.err, ERR_INDEX); return; }
  float2* a = reinterpret_cast<float2*>(c.acc) + 3 * (v.bin_base + pixel);
  float2 ax = a[0], ay = a[1], az = a[2];
  unsigned long long hsum = 0ull;
  for (int k = i; s < v.spp && k < n; ++k, ++s) {
    float4 r = k < i0 + RESOLVE_BLOCK ? srad[k - i0] : c.e.rad[k];
    kahan_add(ax, r.x); kahan_add(ay, r.y); kahan_add(az, r.z);
    if (c.sig) hsum += c.e.sig[k];
  }
  a[0] = ax; a[1] = ay; a[2] = az;
  if (c.sig) c.sacc[v.bin_base + pixel] += hsum;
}

// ------------------------------------------------------------------ gradient scatter
// Lanes holding values for the same key are summed by the lowest such lane
// (peers found with match.any), which then issues the atomics.
template <int NV>
__device__ __forceinline__ void warp_reduce_peers(int key, float (&vals)[NV], float* scratch, bool& leader) {
  int lane = threadIdx.x & 31;
  unsigned peers = __match_any_sync(FULL, key);
#pragma unroll
  for (int k = 0; k < NV; ++k) scratch[lane * (NV + 1) + k] = vals[k];
  __syncwarp();
  leader = key >= 0 && lane == __ffs(peers) - 1;
  if (leader) {
    unsigned rest = peers & ~(1u << lane);
    while (rest) {
      int l = __ffs(rest) - 1;
      rest &= rest - 1;
#pragma unroll
      for (int k = 0; k < NV; ++k) vals[k] += scratch[l * (NV + 1) + k];
    }
  }
  __syncwarp();
}

constexpr int ADJ_BLOCK = 128;

// SMOOTH: interpolated shading normals (SMOOTH); the flat variant keeps its registers
template <bool SMOOTH>
__global__ void __launch_bounds__(ADJ_BLOCK) k_adjoint(KCtx c, long long j0, int n) {
  __shared__ float scratch[ADJ_BLOCK / 32][32 * 17];
  float* scr = scratch[threadIdx.x >> 5];
  const Engine& E = c.e;
  const size_t Q = (size_t)E.Q;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  float* dV = c.args->dV;
  float* dF = c.args->dF;
  int nbv = 0, vi = 0;
  float3 g = mk3(0, 0, 0);
  if (i < n) {
    long long job = j0 + i;
    int si = find_seg(c.segs, c.n_segs, job);
    if (si >= 0) {
      Seg sg = c.segs[si];
      long long local = job - sg.base;
      if (sg.kind == 0 && local < sg.count) {
        DevView v = c.views[sg.view];
        vi = sg.view;
        long long pixel = local / v.spp;
        const float* gp = c.args->dLdI + 3 * (v.pix_off + pixel);
        float inv = 1.0f / (float)v.spp;
        g = mk3(gp[0] * inv, gp[1] * inv, gp[2] * inv);
        if (g.x != 0.0f || g.y != 0.0f || g.z != 0.0f) nbv = E.nb[i];
      }
    }
  }
  // forward sweep: throughput before each vertex
  float3 T[MAX_B];
  T[0] = mk3(1, 1, 1);
  for (int b = 0; b + 1 < nbv; ++b) {
    float4 r0 = E.r0[b * Q + i], r1 = E.r1[b * Q + i], r1n = E.r1[(b + 1) * Q + i];
    int f = __float_as_int(r0.w);
    float3 v0 = fetch_vertex(c.V, c.F[3 * f]), v1 = fetch_vertex(c.V, c.F[3 * f + 1]),
           v2 = fetch_vertex(c.V, c.F[3 * f + 2]);
    float3 wo = -xyz(r1);
    float3 ng = norm3(cross3(v1 - v0, v2 - v0));
    float sg = dot3(ng, wo) < 0.0f ? -1.0f : 1.0f;
    float3 nn = SMOOTH ? shading_normal(c, f, xyz(r0), v0, v1, v2, sg) : ng * sg;
    int tex = __float_as_int(E.r3[b * Q + i].w);
    float3 Qv = brdf_cos(c.brdf, c.fresnel, fetch_mat(c.P, tex), nn, xyz(r1n), wo);
    T[b + 1] = mul(T[b], Qv) * (1.0f / r1n.w);
  }
  bool esc = nbv > 0 && E.esc[i].w != 0.0f;
  float3 A = mk3(0, 0, 0);
  if (esc) A = mul(g, xyz(E.esc[i]));
  float3 Pnext = mk3(0, 0, 0);
  for (int b = c.B - 1; b >= 0; --b) {
    float vals[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) vals[k] = 0.0f;
    int face = -1, key = -1;      // key = texel: equal keys share face and parameters
    if (b < nbv) {
      float4 r0 = E.r0[b * Q + i], r1 = E.r1[b * Q + i], r2 = E.r2[b * Q + i], r3 = E.r3[b * Q + i];
      int f = __float_as_int(r0.w);
      face = f;
      key = __float_as_int(r3.w);
      float3 p = xyz(r0), d = xyz(r1), wo = -d;
      float3 v0 = fetch_vertex(c.V, c.F[3 * f]), v1 = fetch_vertex(c.V, c.F[3 * f + 1]),
             v2 = fetch_vertex(c.V, c.F[3 * f + 2]);
      float3 e1 = v1 - v0, e2 = v2 - v0;
      float3 mv = cross3(e1, e2);
      float ml = len3(mv);
      float3 mh = mv * (1.0f / ml);
      float sgn = dot3(mh, wo) < 0.0f ? -1.0f : 1.0f;
      float3 nn = mh * sgn;
      // with smooth normals: n_s = sgn s / |s|, s = (1 - b1 - b2) N0 + b1 N1 + b2 N2
      float3 N0 = mk3(0, 0, 0), N1 = N0, N2 = N0, sv = N0;
      float b1 = 0.0f, b2 = 0.0f;
      if (SMOOTH) {
        float3 q = p - v0;
        float mm = dot3(mv, mv);
        b1 = dot3(cross3(q, e2), mv) / mm;
        b2 = dot3(cross3(e1, q), mv) / mm;
        N0 = xyz(c.vn[c.F[3 * f]]); N1 = xyz(c.vn[c.F[3 * f + 1]]); N2 = xyz(c.vn[c.F[3 * f + 2]]);
        sv = N0 * (1.0f - b1 - b2) + N1 * b1 + N2 * b2;
        nn = norm3(sv) * sgn;
      }
      Mat m = fetch_mat(c.P, key);
      float3 Nb = mk3(0, 0, 0), Pb = Pnext;
      if (c.sec) Pb += xyz(E.pinj[b * Q + i]);   // the vertex's secondary edge sample moves with p
      float dm[7] = {0, 0, 0, 0, 0, 0, 0};
      float3 gC = mul(g, T[b]);
      float3 C = mk3(0, 0, 0);
      int flags = __float_as_int(r2.w);
      for (int j = 0; j < c.nlt; ++j) {
        if (!(flags & (1 << j))) continue;
        float4 lp, li;
        point_light(c, vi, j, lp, li);
        float3 l = xyz(lp) - p;
        float r = len3(l);
        float3 wi = l * (1.0f / r);
        float ir2 = 1.0f / (r * r);
        float3 Qv = brdf_cos(c.brdf, c.fresnel, m, nn, wi, wo);
        C += mul(Qv, xyz(li)) * ir2;
        float3 gw = mul(gC, xyz(li)) * ir2;
        float3 dwi = mk3(0, 0, 0);
        brdf_cos_adj(c.brdf, c.fresnel, m, nn, wi, wo, gw, Nb, &dwi, dm);
        float sr = gC.x * Qv.x * li.x + gC.y * Qv.y * li.y + gC.z * Qv.z * li.z;
        float rbar = sr * (-2.0f * ir2 / r);
        float3 lbar = (dwi - wi * dot3(dwi, wi)) * (1.0f / r) + wi * rbar;
        Pb -= lbar;
      }
      if (flags & ENV_VIS) {
        float3 wi = xyz(r2), sc = xyz(r3);
        C += mul(brdf_cos(c.brdf, c.fresnel, m, nn, wi, wo), sc);
        brdf_cos_adj(c.brdf, c.fresnel, m, nn, wi, wo, mul(gC, sc), Nb, nullptr, dm);
      }
      float3 w = mk3(0, 0, 0);
      if (b + 1 < nbv || esc) {
        float4 r1n = E.r1[(b + 1) * Q + i];
        float ip = 1.0f / r1n.w;
        float3 wi = xyz(r1n);
        w = brdf_cos(c.brdf, c.fresnel, m, nn, wi, wo) * ip;
        brdf_cos_adj(c.brdf, c.fresnel, m, nn, wi, wo, mul(A, T[b]) * ip, Nb, nullptr, dm);
      }
      A = mul(g, C) + mul(A, w);
      // n = sgn * m / |m|, p = o + t d with t = ((v0 - o) . m) / (d . m)
      float3 mbar, e1d = mk3(0, 0, 0), e2d = mk3(0, 0, 0), qbar = mk3(0, 0, 0);
      if (SMOOTH) {
        // n_s: to the vertex normals (dN, mapped to the vertices around them after
        // the sweep) and to the barycentric weights b1 = q.(e2 x m)/M, b2 =
        // q.(m x e1)/M, q = p - v0, M = m.m
        float sl = len3(sv);
        float3 sh = sv * (1.0f / sl);
        float3 sbar = (Nb - sh * dot3(Nb, sh)) * (sgn / sl);
        float3 g0 = sbar * (1.0f - b1 - b2), g1 = sbar * b1, g2 = sbar * b2;
        float* dN = c.dN + 3 * (size_t)c.F[3 * f];
        atomicAdd(dN, g0.x); atomicAdd(dN + 1, g0.y); atomicAdd(dN + 2, g0.z);
        dN = c.dN + 3 * (size_t)c.F[3 * f + 1];
        atomicAdd(dN, g1.x); atomicAdd(dN + 1, g1.y); atomicAdd(dN + 2, g1.z);
        dN = c.dN + 3 * (size_t)c.F[3 * f + 2];
        atomicAdd(dN, g2.x); atomicAdd(dN + 1, g2.y); atomicAdd(dN + 2, g2.z);
        float b1b = dot3(sbar, N1 - N0), b2b = dot3(sbar, N2 - N0);
        float3 q = p - v0;
        float iM = 1.0f / dot3(mv, mv);
        qbar = (cross3(e2, mv) * b1b + cross3(mv, e1) * b2b) * iM;
        e2d = cross3(mv, q) * (b1b * iM);
        e1d = cross3(q, mv) * (b2b * iM);
        mbar = ((cross3(q, e2) - mv * (2.0f * b1)) * b1b + (cross3(e1, q) - mv * (2.0f * b2)) * b2b) * iM;
        Pb += qbar;
      } else {
        mbar = (Nb - mh * dot3(Nb, mh)) * (sgn / ml);
      }
      float dmv = dot3(d, mv);
      float tb = dot3(Pb, d) / dmv;
      float3 obar = Pb - mv * tb;
      float3 v0bar = mv * tb - qbar;
      mbar += (v0 - p) * tb;
      float3 e1bar = cross3(e2, mbar) + e1d, e2bar = cross3(mbar, e1) + e2d;
      v0bar -= e1bar + e2bar;
      Pnext = obar;
      vals[0] = v0bar.x; vals[1] = v0bar.y; vals[2] = v0bar.z;
      vals[3] = e1bar.x; vals[4] = e1bar.y; vals[5] = e1bar.z;
      vals[6] = e2bar.x; vals[7] = e2bar.y; vals[8] = e2bar.z;
#pragma unroll
      for (int k = 0; k < 7; ++k) vals[9 + k] = dm[k];
    }
    bool leader;
    warp_reduce_peers<16>(key, vals, scr, leader);
    if (leader) {
      if (dV) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          int vid = c.F[3 * face + k];
          atomicAdd(&dV[3 * vid], vals[3 * k]);
          atomicAdd(&dV[3 * vid + 1], vals[3 * k + 1]);
          atomicAdd(&dV[3 * vid + 2], vals[3 * k + 2]);
        }
      }
      if (dF) {
        if (c.np == 7) {
#pragma unroll
          for (int k = 0; k < 7; ++k) atomicAdd(&dF[7 * key + k], vals[9 + k]);
        } else {   // one specular value for all channels: its derivative is the channels' sum
          atomicAdd(&dF[5 * key], vals[9]); atomicAdd(&dF[5 * key + 1], vals[10]); atomicAdd(&dF[5 * key + 2], vals[11]);
          atomicAdd(&dF[5 * key + 3], vals[12] + vals[13] + vals[14]);
          atomicAdd(&dF[5 * key + 4], vals[15]);
        }
      }
    }
  }
}

// Adjoint of the vertex normals after the sweeps (smooth normals): N_v = M_v /
// |M_v| gives Mbar_v = (Nbar_v - N_v (N_v . Nbar_v)) / |M_v| (in place in dN);
// then each face's e1 x e2, a term of the M_v of its three vertices, takes the
// sum of their Mbar and passes it to its vertices.
__global__ void k_vn_adj_vertex(KCtx c) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < c.nv; v += gridDim.x * blockDim.x) {
    float* g = c.dN + 3 * (size_t)v;
    float3 Nb = mk3(g[0], g[1], g[2]);
    float4 n4 = c.vn[v];
    float3 N = xyz(n4);
    float3 Mb = n4.w > 0.0f ? (Nb - N * dot3(N, Nb)) * (1.0f / n4.w) : mk3(0, 0, 0);
    g[0] = Mb.x; g[1] = Mb.y; g[2] = Mb.z;
  }
}

__global__ void k_vn_adj_face(KCtx c) {
  float* dV = c.args->dV;
  if (!dV) return;
  for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < c.nf; f += gridDim.x * blockDim.x) {
    int a = c.F[3 * f], b = c.F[3 * f + 1], d = c.F[3 * f + 2];
    float3 cb = mk3(c.dN[3 * a], c.dN[3 * a + 1], c.dN[3 * a + 2]) +
                mk3(c.dN[3 * b], c.dN[3 * b + 1], c.dN[3 * b + 2]) +
                mk3(c.dN[3 * d], c.dN[3 * d + 1], c.dN[3 * d + 2]);
    float3 v0 = fetch_vertex(c.V, a);
    float3 e1 = fetch_vertex(c.V, b) - v0, e2 = fetch_vertex(c.V, d) - v0;
    float3 e1b = cross3(e2, cb), e2b = cross3(cb, e1), e0b = -(e1b + e2b);
    atomicAdd(&dV[3 * b], e1b.x); atomicAdd(&dV[3 * b + 1], e1b.y); atomicAdd(&dV[3 * b + 2], e1b.z);
    atomicAdd(&dV[3 * d], e2b.x); atomicAdd(&dV[3 * d + 1], e2b.y); atomicAdd(&dV[3 * d + 2], e2b.z);
    atomicAdd(&dV[3 * a], e0b.x); atomicAdd(&dV[3 * a + 1], e0b.y); atomicAdd(&dV[3 * a + 2], e0b.z);
  }
}

__global__ void __launch_bounds__(ADJ_BLOCK) k_edge_resolve(KCtx c, long long j0, int n) {
  __shared__ float scratch[ADJ_BLOCK / 32][32 * 7];
  float* scr = scratch[threadIdx.x >> 5];
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  float vals[6] = {0, 0, 0, 0, 0, 0};
  int key = -1, va = 0, vb = 0;
  if (i < n) {
    long long job = j0 + i;
    int si = find_seg(c.segs, c.n_segs, job);
    if (si >= 0) {
      Seg sg = c.segs[si];
      long long local = job - sg.base;
      long long k = (local >> 6) * 32 + (local & 31);
      if (sg.kind == 1 && local < sg.count && (local & 32) == 0 && k < sg.n_samples) {
        DevView v = c.views[sg.view];
        Key kk{c.args->k0, c.args->k1};
        EdgeSample es = edge_sample(c, sg.view, v, k, sg.n_samples, kk);
        if (es.valid) {
          const float* gp = c.args->dLdI + 3 * (v.pix_off + (long long)es.py * v.W + es.px);
          float3 Lm = xyz(c.e.rad[i]), Lp = xyz(c.e.rad[i + 32]);
          float gsum = gp[0] * (Lm.x - Lp.x) + gp[1] * (Lm.y - Lp.y) + gp[2] * (Lm.z - Lp.z);
          if (gsum != 0.0f) {
            float wt = gsum * (float)c.edge_ncand[sg.view] * es.len / (float)sg.n_samples;
            int2 ev = c.edge_v[es.e];
            float3 ja = cam_project_jt(v, fetch_vertex(c.V, ev.x), es.ns.x, es.ns.y) * (wt * (1.0f - es.tau));
            float3 jb = cam_project_jt(v, fetch_vertex(c.V, ev.y), es.ns.x, es.ns.y) * (wt * es.tau);
            vals[0] = ja.x; vals[1] = ja.y; vals[2] = ja.z;
            vals[3] = jb.x; vals[4] = jb.y; vals[5] = jb.z;
            key = es.e;
            va = ev.x;
            vb = ev.y;
          }
        }
      }
    }
  }
  bool leader;
  warp_reduce_peers<6>(key, vals, scr, leader);
  if (leader) {
    float* dV = c.args->dV;
    atomicAdd(&dV[3 * va], vals[0]); atomicAdd(&dV[3 * va + 1], vals[1]); atomicAdd(&dV[3 * va + 2], vals[2]);
    atomicAdd(&dV[3 * vb], vals[3]); atomicAdd(&dV[3 * vb + 1], vals[4]); atomicAdd(&dV[3 * vb + 2], vals[5]);
  }
}

// ------------------------------------------------------------------ secondary-visibility edges
// At a path vertex p the estimator integrates g(w) = f cos L_in(w) over
// incoming directions; g jumps where w crosses the image of a mesh edge on p's
// sphere of directions, and moving the edge's endpoints (x) or p moves that arc
// by m.(dx - dp)/r along its unit normal m (the boundary term of Li et al.'s
// edge sampling, which the paper's gradient relies on, Sec. 3.2). One sample
// per vertex: an edge picked uniformly from all E edges by an integer map, a
// point x uniform on the part of it above the tangent plane, two side paths at
// w -+ SEC_EPS m that continue the path from the next vertex. Arc length per
// unit edge length is |w x t|/r (t the unit edge direction), so the sample's
// weight is |w x t| E len (tau1 - tau0) / r^2 and its derivative
// <dL/dI, T (g- - g+)> weight m.(dx - dp), dx = (1 - tau) dA + tau dB.
constexpr float SEC_EPS = 1e-4f;    // side rays' angular offset (radians)
constexpr float SEC_BAND = 1e-5f;   // plane-distance band, times (1 + |p|_inf): coplanar faces and edges
constexpr float SEC_RMIN = 1e-6f;   // nearest edge point accepted
constexpr float SEC_SMIN = 1e-6f;   // sine of the edge/view angle accepted

__device__ __forceinline__ float face_side(const KCtx& c, int f, float3 p) {
  float3 a = fetch_vertex(c.V, c.F[3 * f]);
  float3 m = norm3(cross3(fetch_vertex(c.V, c.F[3 * f + 1]) - a, fetch_vertex(c.V, c.F[3 * f + 2]) - a));
  return dot3(m, p - a);
}

// Hierarchy over the edges (importance pick of the secondary edge, Li et al.,
// Sec. 3.2): leaf i holds edges [i G, (i + 1) G) in edge order, with the box of
// their endpoints and their summed length; internal node k unites 2k and 2k + 1.
// Rebuilt by every call that samples with it (the vertices may have moved).
__device__ __forceinline__ float3 face_unit_normal(const KCtx& c, int f) {
  float3 a = fetch_vertex(c.V, c.F[3 * f]);
  return norm3(cross3(fetch_vertex(c.V, c.F[3 * f + 1]) - a, fetch_vertex(c.V, c.F[3 * f + 2]) - a));
}

__global__ void k_etree_leaves(KCtx c, float4* lo, float4* hi, float4* cn) {
  const int nleaf = 1 << c.et_L;
  const float INF = __int_as_float(0x7f800000);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nleaf; i += gridDim.x * blockDim.x) {
    float3 l = mk3(INF, INF, INF), h = mk3(-INF, -INF, -INF), sum = mk3(0, 0, 0);
    float S = 0.0f;
    bool bounded = true;
    int e0 = i * c.et_G, e1 = min(c.n_edges, (i + 1) * c.et_G);
    for (int e = e0; e < e1; ++e) {
      int2 ev = c.edge_v[e];
      float3 a = fetch_vertex(c.V, ev.x), b = fetch_vertex(c.V, ev.y);
      l = mk3(fminf(l.x, fminf(a.x, b.x)), fminf(l.y, fminf(a.y, b.y)), fminf(l.z, fminf(a.z, b.z)));
      h = mk3(fmaxf(h.x, fmaxf(a.x, b.x)), fmaxf(h.y, fmaxf(a.y, b.y)), fmaxf(h.z, fmaxf(a.z, b.z)));
      S += len3(b - a);
      int2 ef = c.edge_f[e];
      if (ef.y < 0) { bounded = false; continue; }
      sum += face_unit_normal(c, ef.x) + face_unit_normal(c, ef.y);
    }
    float4 cone = make_float4(0, 0, 0, -2.0f);
    float sl = len3(sum);
    if (S > 0.0f && bounded && sl > 1e-6f) {
      float3 ax = sum * (1.0f / sl);
      float ct = 1.0f;
      for (int e = e0; e < e1; ++e) {
        int2 ef = c.edge_f[e];
        ct = fminf(ct, fminf(dot3(ax, face_unit_normal(c, ef.x)), dot3(ax, face_unit_normal(c, ef.y))));
      }
      cone = make_float4(ax.x, ax.y, ax.z, ct > 0.0f ? ct : -2.0f);
    }
    lo[nleaf + i] = make_float4(l.x, l.y, l.z, S);
    hi[nleaf + i] = make_float4(h.x, h.y, h.z, 0.0f);
    cn[nleaf + i] = cone;
  }
}

// nodes [2^level, 2^(level+1)) from their children: union of the boxes, sum of
// the lengths, the cone around the normalised sum of the children's axes that
// holds both
__global__ void k_etree_level(float4* lo, float4* hi, float4* cn, int level) {
  const int n = 1 << level;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int k = n + i;
    float4 la = lo[2 * k], lb = lo[2 * k + 1], ha = hi[2 * k], hb = hi[2 * k + 1];
    lo[k] = make_float4(fminf(la.x, lb.x), fminf(la.y, lb.y), fminf(la.z, lb.z), la.w + lb.w);
    hi[k] = make_float4(fmaxf(ha.x, hb.x), fmaxf(ha.y, hb.y), fmaxf(ha.z, hb.z), 0.0f);
    float4 ca = cn[2 * k], cb = cn[2 * k + 1];
    float4 cone = make_float4(0, 0, 0, -2.0f);
    if (!(la.w > 0.0f) || !(lb.w > 0.0f)) {
      cone = la.w > 0.0f ? ca : cb;
    } else if (ca.w > -1.5f && cb.w > -1.5f) {
      float3 sum = xyz(ca) + xyz(cb);
      float sl = len3(sum);
      if (sl > 1e-6f) {
        float3 ax = sum * (1.0f / sl);
        auto ang = [](float x) { return acosf(fmaxf(-1.0f, fminf(1.0f, x))); };
        float th = fmaxf(ang(dot3(ax, xyz(ca))) + ang(ca.w), ang(dot3(ax, xyz(cb))) + ang(cb.w));
        cone = make_float4(ax.x, ax.y, ax.z, th < 0.5f * PI_F ? cosf(th) : -2.0f);
      }
    }
    cn[k] = cone;
  }
}

// Importance of node k at a vertex (p, tangent-plane normal n, band bnd): 0 when
// its box lies at or below the plane or, sampling silhouettes, when every face on
// its edges sees p on the same side (n_f.(p - x) within |v| cos(phi -+ th) -+ r
// over the box and the cone: v = p - centre, r the half-diagonal, phi the angle
// of v to the axis, th the cone's half-angle); else summed length / max(d^2,
// diag^2 / 4), d the distance from p to the box.
__device__ __forceinline__ float etree_weight(const KCtx& c, int k, float3 p, float3 n, float bnd) {
  float4 lo = c.et_lo[k], hi = c.et_hi[k];
  if (!(lo.w > 0.0f)) return 0.0f;
  float top = (n.x > 0.0f ? hi.x - p.x : lo.x - p.x) * n.x + (n.y > 0.0f ? hi.y - p.y : lo.y - p.y) * n.y +
              (n.z > 0.0f ? hi.z - p.z : lo.z - p.z) * n.z;
  if (!(top > bnd)) return 0.0f;
  if (c.edge_mode == 0) {
    float4 cn = c.et_cn[k];
    if (cn.w > -1.5f) {
      float3 v = p - (xyz(lo) + xyz(hi)) * 0.5f;
      float r = 0.5f * len3(xyz(hi) - xyz(lo)), D = len3(v);
      if (D > r) {
        float cp = dot3(xyz(cn), v) / D, sp = sqrtf(fmaxf(0.0f, 1.0f - cp * cp));
        float cq = cn.w, sq = sqrtf(fmaxf(0.0f, 1.0f - cq * cq));
        float cmin = cp <= -cq ? -1.0f : cp * cq - sp * sq;
        float cmax = cp >= cq ? 1.0f : cp * cq + sp * sq;
        if (D * cmin - r > -bnd || D * cmax + r < bnd) return 0.0f;
      }
    }
  }
  float dx = fmaxf(lo.x - p.x, fmaxf(0.0f, p.x - hi.x)), dy = fmaxf(lo.y - p.y, fmaxf(0.0f, p.y - hi.y)),
        dz = fmaxf(lo.z - p.z, fmaxf(0.0f, p.z - hi.z));
  float ex = hi.x - lo.x, ey = hi.y - lo.y, ez = hi.z - lo.z;
  float den = fmaxf(dx * dx + dy * dy + dz * dz, 0.25f * (ex * ex + ey * ey + ez * ez));
  return lo.w / fmaxf(den, 1e-30f);
}

struct SecSample {
  int e;
  float tau, weight;
  float3 w, mh;
};

// Edge sample at vertex p (shading normal n, face f0): false if the picked edge
// is not a candidate (an edge of f0, not a silhouette seen from p in
// silhouette mode, or wholly at or below the tangent plane).
// ct, b, key: the vertex's counters, for the hierarchy's per-level uniforms
// (draw (c0, c1, b<<4 | (4 + j/4), stream), word j % 4 at level j)
__device__ __forceinline__ bool sec_sample(const KCtx& c, float3 p, float3 n, float3 ns, int f0, uint32_t u0,
                                           uint32_t u1, int4 ct, int b, Key key, SecSample& s) {
  int nE = c.n_edges;
  if (nE <= 0) return false;
  float bnd = SEC_BAND * (1.0f + fmaxf(fabsf(p.x), fmaxf(fabsf(p.y), fabsf(p.z))));
  float inv_p;   // 1 / pick probability
  if (c.sec_tree) {
    int k = 1;
    float pr = 1.0f;
    U4 u = {0, 0, 0, 0};
    for (int j = 0; j < c.et_L; ++j) {
      if ((j & 3) == 0)
        u = philox((uint32_t)ct.x, (uint32_t)ct.y, (uint32_t)(b << 4) | (4u + (uint32_t)(j >> 2)), (uint32_t)ct.z,
                   key.k0, key.k1);
      uint32_t w = (j & 3) == 0 ? u.x : (j & 3) == 1 ? u.y : (j & 3) == 2 ? u.z : u.w;
      float wa = etree_weight(c, 2 * k, p, n, bnd), wb = etree_weight(c, 2 * k + 1, p, n, bnd);
      if (!(wa + wb > 0.0f)) return false;
      if (unif(w) < wa / (wa + wb)) { k = 2 * k; pr *= wa / (wa + wb); }
      else { k = 2 * k + 1; pr *= wb / (wa + wb); }
    }
    int first = (k - (1 << c.et_L)) * c.et_G;
    int cnt = min(c.et_G, nE - first);
    if (cnt <= 0) return false;
    pr /= (float)cnt;
    s.e = first + (int)(((unsigned long long)(u0 >> 8) * (unsigned long long)cnt) >> 24);
    inv_p = 1.0f / pr;
  } else {
    s.e = (int)(((unsigned long long)(u0 >> 8) * (unsigned long long)nE) >> 24);
    inv_p = (float)nE;
  }
  int2 ef = c.edge_f[s.e];
  if (ef.x == f0 || ef.y == f0) return false;
  if (c.edge_mode == 0) {
    float s1 = face_side(c, ef.x, p);
    bool sil;
    if (ef.y >= 0) {
      float s2 = face_side(c, ef.y, p);
      sil = (s1 > bnd && s2 < -bnd) || (s1 < -bnd && s2 > bnd);
    } else {
      sil = fabsf(s1) > bnd;
    }
    if (!sil) return false;
  }
  int2 ev = c.edge_v[s.e];
  float3 A = fetch_vertex(c.V, ev.x), Bv = fetch_vertex(c.V, ev.y);
  // the part above the tangent plane (and, with shading normals, above the
  // shading plane too)
  float t0 = 0.0f, t1 = 1.0f;
  for (int pl = 0; pl < (c.smooth ? 2 : 1); ++pl) {
    float3 nc = pl == 0 ? n : ns;
    float hA = dot3(nc, A - p), hB = dot3(nc, Bv - p);
    if (!(hA > bnd) && !(hB > bnd)) return false;
    if (!(hA > bnd)) t0 = fmaxf(t0, (bnd - hA) / (hB - hA));
    if (!(hB > bnd)) t1 = fminf(t1, (hA - bnd) / (hA - hB));
  }
  if (!(t1 > t0)) return false;
  s.tau = t0 + unif(u1) * (t1 - t0);
  float3 tv = Bv - A;
  float3 dv = A + tv * s.tau - p;
  float r = len3(dv);
  if (!(r > SEC_RMIN)) return false;
  s.w = dv * (1.0f / r);
  float l = len3(tv);
  float3 cr = cross3(s.w, tv * (1.0f / l));
  float sn = len3(cr);
  if (!(sn > SEC_SMIN)) return false;
  s.mh = cr * (1.0f / sn);
  s.weight = sn * inv_p * l * (t1 - t0) / (r * r);
  return true;
}

// normals of a recorded vertex at p on face f: the face normal turned toward
// wo (n) and the shading normal (ns: n, or interpolated)
__device__ __forceinline__ void vertex_normals(const KCtx& c, int f, float3 p, float3 wo, float3& n, float3& ns) {
  float3 v0 = fetch_vertex(c.V, c.F[3 * f]), v1 = fetch_vertex(c.V, c.F[3 * f + 1]),
         v2 = fetch_vertex(c.V, c.F[3 * f + 2]);
  float3 ng = norm3(cross3(v1 - v0, v2 - v0));
  float sgn = dot3(ng, wo) < 0.0f ? -1.0f : 1.0f;
  n = ng * sgn;
  ns = c.smooth ? shading_normal(c, f, p, v0, v1, v2, sgn) : n;
}

// One edge sample per recorded vertex of every camera path of the chunk whose
// pixel has a nonzero dL/dI; accepted samples become jobs.
__global__ void __launch_bounds__(ADJ_BLOCK) k_sec_gen(KCtx c, long long j0, int n) {
  const Engine& E = c.e;
  const size_t Q = (size_t)E.Q;
  const long long cap = E.sec_cap;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int nbv = 0;
  float3 g = mk3(0, 0, 0);
  if (i < n) {
    long long job = j0 + i;
    int si = find_seg(c.segs, c.n_segs, job);
    if (si >= 0) {
      Seg sg = c.segs[si];
      long long local = job - sg.base;
      if (sg.kind == 0 && local < sg.count) {
        DevView v = c.views[sg.view];
        long long pixel = local / v.spp;
        const float* gp = c.args->dLdI + 3 * (v.pix_off + pixel);
        float inv = 1.0f / (float)v.spp;
        g = mk3(gp[0] * inv, gp[1] * inv, gp[2] * inv);
        if (g.x != 0.0f || g.y != 0.0f || g.z != 0.0f) nbv = E.nb[i];
      }
    }
  }
  Key key{c.args->k0, c.args->k1};
  int4 ct = nbv > 0 ? E.ctr[i] : make_int4(0, 0, 0, 0);
  float3 T = mk3(1, 1, 1);
  int made = 0;
  for (int b = 0; b < c.B; ++b) {
    bool ok = false;
    SecSample ss;
    float4 r0 = make_float4(0, 0, 0, 0);
    float3 Tn = T;
    if (b < nbv) {
      r0 = E.r0[b * Q + i];
      float4 r1 = E.r1[b * Q + i];
      int f = __float_as_int(r0.w);
      float3 wo = -xyz(r1);
      float3 nn, ns;
      vertex_normals(c, f, xyz(r0), wo, nn, ns);
      E.pinj[b * Q + i] = make_float4(0, 0, 0, 0);
      U4 u = philox((uint32_t)ct.x, (uint32_t)ct.y, (uint32_t)(b << 4) | 3u, (uint32_t)ct.z, key.k0, key.k1);
      ok = sec_sample(c, xyz(r0), nn, ns, f, u.x, u.y, ct, b, key, ss);
      if (b + 1 < nbv) {
        float4 r1n = E.r1[(b + 1) * Q + i];
        int tex = __float_as_int(E.r3[b * Q + i].w);
        Tn = mul(T, brdf_cos(c.brdf, c.fresnel, fetch_mat(c.P, tex), ns, xyz(r1n), wo)) * (1.0f / r1n.w);
      }
    }
    int q = warp_append(&E.cnt[CNT_SEC], ok);
    if (ok && q < cap) {
      float3 gC = mul(g, T);
      E.sj[q] = r0;
      E.sj[cap + q] = make_float4(ss.w.x, ss.w.y, ss.w.z, ss.weight);
      E.sj[2 * cap + q] = make_float4(ss.mh.x, ss.mh.y, ss.mh.z, ss.tau);
      E.sj[3 * cap + q] = make_float4(gC.x, gC.y, gC.z, __int_as_float(ss.e));
      E.sje[q] = make_int4(ct.x, ct.y, i, b | (ct.w & ~15));
      ++made;
    }
    T = Tn;
  }
  for (int off = 16; off > 0; off >>= 1) made += __shfl_xor_sync(FULL, made, off);
  if ((threadIdx.x & 31) == 0 && made) atomicAdd(&E.stat[STAT_SEC], (unsigned long long)made);
}

// Side-index space of J jobs (blocks of 64: 32 minus sides, then their plus
// sides) that falls into pass `pass` (slots [0, n) of the engine); 0 when the
// pass has no work, so empty passes of a captured graph cost one launch each.
__device__ __forceinline__ int sec_pass_slots(const Engine& E, int pass, long long& J) {
  J = min((long long)E.cnt[CNT_SEC], E.sec_cap);
  long long rest = (J + 31) / 32 * 64 - (long long)pass * E.Q;
  return (int)max(0LL, min(rest, (long long)E.Q));
}

// Side paths of pass `pass`: side index s = pass * Q + slot. Grid-stride over
// the pass's slots.
__global__ void k_sec_raygen(KCtx c, int pass) {
  const Engine& E = c.e;
  const size_t Q = (size_t)E.Q;
  const long long cap = E.sec_cap;
  long long J;
  const int total = sec_pass_slots(E, pass, J);
  for (int base = blockIdx.x * blockDim.x; base < total; base += gridDim.x * blockDim.x) {
    int i = base + threadIdx.x;
    long long sidx = (long long)pass * E.Q + i;
    long long job = (sidx >> 6) * 32 + (sidx & 31);
    bool ok = false;
    if (i < total && job < J) {
      float4 a = E.sj[job], w = E.sj[cap + job], m = E.sj[2 * cap + job];
      int4 je = E.sje[job];
      int slot = je.z, b = je.w & 15, f = __float_as_int(a.w);
      float3 wo = -xyz(E.r1[b * Q + slot]);
      float3 nn, ns;
      vertex_normals(c, f, xyz(a), wo, nn, ns);
      float3 ws = norm3(xyz(w) + xyz(m) * ((sidx & 32) ? SEC_EPS : -SEC_EPS));
      float3 thr = brdf_cos(c.brdf, c.fresnel, fetch_mat(c.P, __float_as_int(E.r3[b * Q + slot].w)), ns, ws, wo);
      if (c.smooth && !(dot3(nn, ws) > 0.0f)) thr = mk3(0, 0, 0);   // below the face
      E.rad[i] = make_float4(0, 0, 0, 0);
      if (thr.x > 0.0f || thr.y > 0.0f || thr.z > 0.0f) {
        E.o[i] = make_float4(a.x, a.y, a.z, 0.0f);
        E.d[i] = make_float4(ws.x, ws.y, ws.z, 0.0f);
        E.thr[i] = make_float4(thr.x, thr.y, thr.z, 0.0f);
        E.origin[i] = f;
        E.ctr[i] = make_int4(je.x, je.y, 16 + b, (b + 1) | (je.w & ~15));
        ok = true;
      }
    }
    int q = warp_append(&E.cnt[CNT_EXT + 0], ok);
    if (ok) E.q0[q] = i;
    unsigned mk = __ballot_sync(FULL, ok);
    if ((threadIdx.x & 31) == 0 && mk) atomicAdd(&E.stat[STAT_PATHS], (unsigned long long)__popc(mk));
  }
}

// (g- - g+) of each job of the pass: edge endpoints get weight (1 - tau, tau)
// times m, the vertex position's adjoint gets -m (read by k_adjoint).
__global__ void __launch_bounds__(ADJ_BLOCK) k_sec_resolve(KCtx c, int pass) {
  __shared__ float scratch[ADJ_BLOCK / 32][32 * 7];
  float* scr = scratch[threadIdx.x >> 5];
  const Engine& E = c.e;
  const size_t Q = (size_t)E.Q;
  const long long cap = E.sec_cap;
  long long J;
  const int total = sec_pass_slots(E, pass, J);
  for (int base = blockIdx.x * blockDim.x; base < total; base += gridDim.x * blockDim.x) {
    int i = base + threadIdx.x;
    long long sidx = (long long)pass * E.Q + i;
    long long job = (sidx >> 6) * 32 + (sidx & 31);
    float vals[6] = {0, 0, 0, 0, 0, 0};
    int key = -1, va = 0, vb = 0;
    if (i < total && (sidx & 32) == 0 && job < J) {
      float3 Lm = xyz(E.rad[i]), Lp = xyz(E.rad[i + 32]);
      float4 w = E.sj[cap + job], m = E.sj[2 * cap + job], gq = E.sj[3 * cap + job];
      float cv = (gq.x * (Lm.x - Lp.x) + gq.y * (Lm.y - Lp.y) + gq.z * (Lm.z - Lp.z)) * w.w;
      if (cv != 0.0f) {
        int4 je = E.sje[job];
        float3 mh = xyz(m);
        int e = __float_as_int(gq.w);
        int2 ev = c.edge_v[e];
        float3 da = mh * (cv * (1.0f - m.w)), db = mh * (cv * m.w);
        vals[0] = da.x; vals[1] = da.y; vals[2] = da.z;
        vals[3] = db.x; vals[4] = db.y; vals[5] = db.z;
        key = e;
        va = ev.x;
        vb = ev.y;
        E.pinj[(je.w & 15) * Q + je.z] = make_float4(-cv * mh.x, -cv * mh.y, -cv * mh.z, 0.0f);
      }
    }
    bool leader;
    warp_reduce_peers<6>(key, vals, scr, leader);
    if (leader) {
      float* dV = c.args->dV;
      atomicAdd(&dV[3 * va], vals[0]); atomicAdd(&dV[3 * va + 1], vals[1]); atomicAdd(&dV[3 * va + 2], vals[2]);
      atomicAdd(&dV[3 * vb], vals[3]); atomicAdd(&dV[3 * vb + 1], vals[4]); atomicAdd(&dV[3 * vb + 2], vals[5]);
    }
  }
}

__global__ void k_reset_pass(int* cnt) {
  for (int i = threadIdx.x; i < CNT_MISC; i += blockDim.x) cnt[i] = 0;
}

// (L- - L+) of each shadow-edge sample: the edge's endpoints move the boundary
// through the light ray (s P^T js), the receiver's vertices through its plane
// (u ds), js = J_proj(q)^T n_S.
__global__ void k_sh_resolve(KCtx c, long long j0, int n) {
  const Engine& E = c.e;
  const size_t Q = (size_t)E.Q;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  long long job = j0 + i;
  int si = find_seg(c.segs, c.n_segs, job);
  if (si < 0) return;
  Seg sg = c.segs[si];
  long long local = job - sg.base;
  if (sg.kind != 2 || local >= sg.count || (local & 32)) return;
  float4 r0 = E.shr[i];
  if (!(r0.x == r0.x)) return;
  DevView v = c.views[sg.view];
  int px = (int)floorf(r0.x), py = (int)floorf(r0.y);
  const float* gp = c.args->dLdI + 3 * (v.pix_off + (long long)py * v.W + px);
  float3 Lm = xyz(E.rad[i]), Lp = xyz(E.rad[i + 32]);
  float g = gp[0] * (Lm.x - Lp.x) + gp[1] * (Lm.y - Lp.y) + gp[2] * (Lm.z - Lp.z);
  if (g == 0.0f) return;
  float4 r1 = E.shr[Q + i], r2 = E.shr[2 * Q + i];
  float wt = g * r2.z;
  float tau = r2.x, sc = r2.w;
  int e = __float_as_int(r2.y), rf = __float_as_int(r1.w);
  float3 q = xyz(r1);
  float4 lp, li;
  point_light(c, sg.view, sg.light, lp, li);
  float3 L = xyz(lp);
  int2 ev = c.edge_v[e];
  float3 A = fetch_vertex(c.V, ev.x), Bv = fetch_vertex(c.V, ev.y);
  float3 uv = A + (Bv - A) * tau - L;
  int f0 = c.F[3 * rf], f1 = c.F[3 * rf + 1], f2 = c.F[3 * rf + 2];
  float3 v0 = fetch_vertex(c.V, f0), v1 = fetch_vertex(c.V, f1), v2 = fetch_vertex(c.V, f2);
  float3 e1 = v1 - v0, e2 = v2 - v0, nr = cross3(e1, e2);
  float nu = dot3(nr, uv);
  float3 js = cam_project_jt(v, q, r0.z, r0.w);
  float3 pj = (js - nr * (dot3(uv, js) / nu)) * (wt * sc);
  float* dV = c.args->dV;
  float3 ga = pj * (1.0f - tau), gb = pj * tau;
  atomicAdd(&dV[3 * ev.x], ga.x); atomicAdd(&dV[3 * ev.x + 1], ga.y); atomicAdd(&dV[3 * ev.x + 2], ga.z);
  atomicAdd(&dV[3 * ev.y], gb.x); atomicAdd(&dV[3 * ev.y + 1], gb.y); atomicAdd(&dV[3 * ev.y + 2], gb.z);
  float kap = wt * dot3(js, uv) / nu;
  float3 w = q - v0;
  float3 c1 = cross3(e2, w), c2 = cross3(w, e1);
  float3 g0 = (nr + c1 + c2) * kap, g1 = c1 * (-kap), g2 = c2 * (-kap);
  atomicAdd(&dV[3 * f0], g0.x); atomicAdd(&dV[3 * f0 + 1], g0.y); atomicAdd(&dV[3 * f0 + 2], g0.z);
  atomicAdd(&dV[3 * f1], g1.x); atomicAdd(&dV[3 * f1 + 1], g1.y); atomicAdd(&dV[3 * f1 + 2], g1.z);
  atomicAdd(&dV[3 * f2], g2.x); atomicAdd(&dV[3 * f2 + 1], g2.y); atomicAdd(&dV[3 * f2 + 2], g2.z);
}

// closest-hit queries for st_trace_closest
__global__ void __launch_bounds__(EXT_BLOCK) k_trace_rays(const float4* nodes, const float4* tri, int nf, int nn,
                                                          const float4* rays, int n, int exclude, int* out_tri,
                                                          float* out_t, int* err) {
  __shared__ int sstack[TRACE_SH * EXT_BLOCK];
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float4 a = rays[2 * i], b = rays[2 * i + 1];
  float t;
  int f = trace_bvh<false, false>(nodes, tri, nf, nn, xyz(a), xyz(b), b.w, exclude, t, sstack + threadIdx.x, err, nullptr);
  out_tri[i] = f;
  out_t[i] = f >= 0 ? t : __int_as_float(0x7f800000);
}

}  // namespace st

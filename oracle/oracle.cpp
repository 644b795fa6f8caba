// FP64 CPU oracle of the differentiable path trace -- TEST INFRASTRUCTURE ONLY.
//
// Only the test suite, the package smoke check and the benchmark's CPU-baseline
// leg may load this library. It shares no code, header, constant table or
// helper with the CUDA library; both are written from the estimator stated
// below, which restates the paper's renderer R(x, m, c) (Sec. 3.2, "Vertex
// optimization") with the material of Sec. 3.3 ("Representation": a
// Torrance-Sparrow BRDF with diffuse albedo, specular and roughness, stored per
// face = mesh colors at r = 0) under point lights or an HDR environment map
// (Sec. 3.1 "Input"), with global illumination (Sec. 3.3 "Effects of Global
// Illumination"; B = 1 is the paper's "local + shadows" case).
//
// ESTIMATOR (the paper names only the model; every convention below is a
// reading, recorded with the others in the design notes):
//  * Random numbers: Philox4x32-10 (Salmon et al., SC'11), key = (seed lo, seed
//    hi). Counter words: camera paths (pixel_offset + y*W + x, sample, b<<4|call,
//    0); edge selection (k, pixel_offset, 0, 1); edge side paths (k,
//    pixel_offset, b<<4|call, 2). Call 0 at b = 0 = pixel jitter, call 1 =
//    environment NEE, call 2 = BSDF sampling. Uniform = (x >> 8) * 2^-24.
//  * Camera: pinhole, fov_y, +y up, row 0 at the top, box-filter jitter.
//  * Intersection: watertight test (Woop, Benthin, Wald, JCGT 2013), closest
//    t in (T_EPS, tmax), origin triangle excluded, equal t -> lower face id.
//  * Shading: flat face normal flipped toward the incoming ray (two-sided); with
//    the scene option smooth_normals, a shading normal interpolated from vertex
//    normals, used for NEE, BRDF, sampling and pdfs, a direction counting only
//    above both planes (see shading_normal).
//  * BRDF: f = kd/pi + F D G1(i) G1(o) / (4 cos_i cos_o) with the "specular
//    color" ks (one value for all channels with 5 parameters per texel, one
//    per channel with 7): the Fresnel factor F is held at its normal-incidence
//    value ks (scene option fresnel = 0, so ks = 0 is exactly Lambertian) or is
//    Schlick's ks + (1 - ks)(1 - wi.h)^5 (fresnel = 1); D = GGX or Beckmann
//    with alpha = roughness (clamped to [0.01, 1]); separable Smith G1.
//  * Lobe choice p_s = clamp(mean ks / (mean ks + mean kd), 0.05, 0.95); diffuse by the
//    concentric-disk (Shirley-Chiu) cosine map, specular by h ~ D cos(theta_h)
//    and reflection, in a tangent frame t = (h x n)/|h x n|, b = n x t about a
//    fixed helper axis h (the lobes are isotropic, so the frame's rotation
//    about n changes no density); pdf = one-sample mixture; invalid (below the
//    surface) ends the path.
//  * NEE: every point light (no MIS); one environment sample per vertex from an
//    alias table (Vose) over texel weight lum * sin(theta_row), MIS power
//    heuristic against the BSDF pdf (weight 1 at the last vertex, which draws no
//    BSDF direction). Escaped BSDF rays collect the environment with the
//    complementary weight; a primary miss collects it unweighted.
//  * B vertices with NEE, no Russian roulette. Pixel = mean over samples.
//  * Interior gradient: derivative of the estimator with sampled directions,
//    pdfs and MIS weights held constant and point-light directions
//    differentiated; computed here with sparse forward-mode dual numbers.
//  * Edge term (primary visibility): candidates = silhouette (or all) edges
//    whose screen projection survives clipping; sample k of N_e picks one with
//    probability 1/n_cand by a stratified integer map (consecutive samples walk
//    the candidate list in order), a point uniformly along its clipped screen
//    segment, trace one path each side at
//    +-EDGE_EPS pixels along the screen normal with shared random numbers, and
//    scatter (L- - L+) <dL/dI_pixel> v_n * n_cand * len / N_e to the two
//    endpoints with screen-space weights (1 - tau, tau).
//  * Edge term (secondary visibility, gradients only, orc_params.secondary):
//    at every vertex b of a camera path, one edge of the mesh picked uniformly
//    (u from counter (c0, c1, b<<4|3, stream): integer pick (u0>>8)*E>>24, u1
//    along the edge; secondary = 2 picks through the edge hierarchy instead, see
//    EdgeTree), kept if it is a silhouette seen from the vertex (or every
//    edge, edge_mode 1), is not an edge of the vertex's face, and has a part
//    above the tangent plane; a point uniform on that part; two side paths at
//    +-SEC_EPS radians across the edge's arc continue the path from vertex
//    b + 1 (counters (c0, c1, vertex<<4|call, 16 + b)); see secondary_edge().
//  * Shadow-edge term (point lights): see orc_shadow_edge_grad.
#include "oracle.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <thread>
#include <type_traits>
#include <vector>

namespace {

constexpr double PI = 3.14159265358979323846;
constexpr double T_EPS = 1e-5;
constexpr double Z_NEAR = 1e-4;
constexpr double EDGE_EPS = 1e-3;
constexpr double SH_EDGE_DELTA = 1e-4;   // shadow edge: receiver search starts this far (relative) past the edge
constexpr double SEC_EPS = 1e-4;     // secondary edge: angular offset of the two side rays (radians)
constexpr double SEC_BAND = 1e-5;    // secondary edge: plane-distance band, times (1 + |p|_inf)
constexpr double SEC_RMIN = 1e-6;    // secondary edge: nearest edge point accepted
constexpr double SEC_SMIN = 1e-6;    // secondary edge: sine of the edge/view angle accepted
constexpr int MAX_B = 8;
constexpr int MAXD = 64 * MAX_B;   // dual dimensions of one path (checked: see Vars)

// ---------------------------------------------------------------- Philox
struct U4 { uint32_t w[4]; };

U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
  // Salmon et al. SC'11: 10 rounds of (mulhilo, xor with key and the other
  // words); the key is bumped by the Weyl constants between rounds.
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += W0; k1 += W1; }
    uint64_t p0 = (uint64_t)M0 * c.w[0];
    uint64_t p1 = (uint64_t)M1 * c.w[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    U4 n = {{hi1 ^ c.w[1] ^ k0, lo1, hi0 ^ c.w[3] ^ k1, lo0}};
    c = n;
  }
  return c;
}

inline double unif(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0); }

// Path signature: FNV-1a style 64-bit hash of a path's discrete decisions, in
// this order at every vertex: the face hit (0xffffffff for a miss), then for a
// miss under an environment the texel its direction reads (nearest lookup),
// for a hit with mesh colors at r > 0 the texel the hit point picks, the
// environment texel drawn for NEE, the BSDF lobe code (1 = specular, + 2 when
// the sampled direction is valid) where a direction is drawn, and the
// visibility bits of the vertex's shadow rays (bit j = point light j seen, bit
// 8 = the environment sample seen) when at least one was traced. A pixel's
// signature is the sum of its samples' hashes modulo 2^64. Equal signatures mean
// the two implementations took the same decisions, so their values may differ
// only by rounding.
constexpr uint64_t SIG_BASIS = 0xcbf29ce484222325ull;
inline uint64_t sig_mix(uint64_t h, uint32_t x) { return (h ^ (uint64_t)x) * 0x100000001b3ull; }

struct Rng {
  uint32_t k0, k1;
  U4 draw(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3) const {
    U4 c = {{c0, c1, c2, c3}};
    return philox4x32_10(c, k0, k1);
  }
};

// ---------------------------------------------------------------- dual numbers
struct Dual {
  double v;
  int n;
  double g[MAXD];
  Dual() : v(0), n(0) {}
  Dual(double x) : v(x), n(0) {}
  Dual(const Dual& o) : v(o.v), n(o.n) { std::memcpy(g, o.g, sizeof(double) * n); }
  Dual& operator=(const Dual& o) {
    v = o.v; n = o.n; std::memcpy(g, o.g, sizeof(double) * n); return *this;
  }
};

inline double vv(double x) { return x; }
inline double vv(const Dual& x) { return x.v; }

// r.g = ca * a.g + cb * b.g
inline void lin2(Dual& r, const Dual& a, double ca, const Dual& b, double cb) {
  r.n = std::max(a.n, b.n);
  for (int k = 0; k < r.n; ++k)
    r.g[k] = (k < a.n ? ca * a.g[k] : 0.0) + (k < b.n ? cb * b.g[k] : 0.0);
}
inline void lin1(Dual& r, const Dual& a, double ca) {
  r.n = a.n;
  for (int k = 0; k < r.n; ++k) r.g[k] = ca * a.g[k];
}
inline Dual operator+(const Dual& a, const Dual& b) { Dual r(a.v + b.v); lin2(r, a, 1, b, 1); return r; }
inline Dual operator-(const Dual& a, const Dual& b) { Dual r(a.v - b.v); lin2(r, a, 1, b, -1); return r; }
inline Dual operator*(const Dual& a, const Dual& b) { Dual r(a.v * b.v); lin2(r, a, b.v, b, a.v); return r; }
inline Dual operator/(const Dual& a, const Dual& b) {
  Dual r(a.v / b.v); lin2(r, a, 1.0 / b.v, b, -a.v / (b.v * b.v)); return r;
}
inline Dual operator-(const Dual& a) { Dual r(-a.v); lin1(r, a, -1); return r; }
inline Dual operator+(const Dual& a, double b) { Dual r(a.v + b); lin1(r, a, 1); return r; }
inline Dual operator+(double b, const Dual& a) { Dual r(b + a.v); lin1(r, a, 1); return r; }
inline Dual operator-(const Dual& a, double b) { Dual r(a.v - b); lin1(r, a, 1); return r; }
inline Dual operator-(double b, const Dual& a) { Dual r(b - a.v); lin1(r, a, -1); return r; }
inline Dual operator*(const Dual& a, double b) { Dual r(a.v * b); lin1(r, a, b); return r; }
inline Dual operator*(double b, const Dual& a) { Dual r(b * a.v); lin1(r, a, b); return r; }
inline Dual operator/(const Dual& a, double b) { Dual r(a.v / b); lin1(r, a, 1.0 / b); return r; }
inline Dual operator/(double b, const Dual& a) { Dual r(b / a.v); lin1(r, a, -b / (a.v * a.v)); return r; }
inline Dual sqrt(const Dual& a) { double s = std::sqrt(a.v); Dual r(s); lin1(r, a, 0.5 / s); return r; }
inline Dual exp(const Dual& a) { double e = std::exp(a.v); Dual r(e); lin1(r, a, e); return r; }
inline Dual erf(const Dual& a) {
  Dual r(std::erf(a.v)); lin1(r, a, 2.0 / std::sqrt(PI) * std::exp(-a.v * a.v)); return r;
}
inline Dual fabs(const Dual& a) { return a.v < 0 ? -a : a; }

using std::sqrt; using std::exp; using std::erf; using std::fabs;

// ---------------------------------------------------------------- vectors
template <class T> struct V3 { T x, y, z; };
template <class T> inline V3<T> mk(T x, T y, T z) { return V3<T>{x, y, z}; }
template <class T> inline V3<T> operator+(const V3<T>& a, const V3<T>& b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
template <class T> inline V3<T> operator-(const V3<T>& a, const V3<T>& b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <class T> inline V3<T> operator-(const V3<T>& a) { return {-a.x, -a.y, -a.z}; }
template <class T, class S> inline V3<T> scl(const V3<T>& a, const S& s) { return {a.x * s, a.y * s, a.z * s}; }
template <class T> inline T dot(const V3<T>& a, const V3<T>& b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <class T> inline V3<T> cross(const V3<T>& a, const V3<T>& b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
template <class T> inline T len(const V3<T>& a) { return sqrt(dot(a, a)); }
template <class T> inline V3<T> nrm(const V3<T>& a) { T l = len(a); return {a.x / l, a.y / l, a.z / l}; }
template <class T> inline V3<T> lift(const V3<double>& a) { return {T(a.x), T(a.y), T(a.z)}; }
template <class T> inline V3<double> val(const V3<T>& a) { return {vv(a.x), vv(a.y), vv(a.z)}; }
using V3d = V3<double>;
inline double comp(const V3d& a, int k) { return k == 0 ? a.x : (k == 1 ? a.y : a.z); }

// ---------------------------------------------------------------- scene
struct Scene {
  int nv = 0, nf = 0;
  int res = 0, ntex = 1;        // mesh-colors resolution r and texels per face (r+1)(r+2)/2
  std::vector<V3d> vert;
  std::vector<int> face;        // 3 per face
  int np = 5;                   // parameters per texel: kd rgb, ks, alpha (5) or kd rgb, ks rgb, alpha (7)
  std::vector<double> param;    // np per texel
  int brdf = 0;
  int fresnel = 0;              // 0: Fresnel factor held at ks; 1: Schlick with F0 = ks
  std::vector<V3d> lpos, lint;
  int ew = 0, eh = 0;
  std::vector<double> env;      // 3 per texel
  std::vector<double> prob, pmf;
  std::vector<int> alias;
  bool smooth = false;          // interpolated shading normals
  std::vector<int> vf_start, vf_list;   // faces around each vertex (CSR, face order)
};

// Point lights a path of one view sees: the scene's, then the view's own
// (e.g. a light at the camera, Sec. 4), in that order.
struct Lights { std::vector<V3d> pos, I; };

struct Cam {
  V3d eye, fwd, right, up;
  double th, aspect;
  int W, H, spp;
  uint32_t off;
  Lights lt;
};

Cam make_cam(const orc_view& v, const Scene& s) {
  Cam c;
  c.lt.pos = s.lpos;
  c.lt.I = s.lint;
  for (int j = 0; j < v.n_lights && j < 2; ++j) {
    c.lt.pos.push_back({v.light_pos[j][0], v.light_pos[j][1], v.light_pos[j][2]});
    c.lt.I.push_back({v.light_intensity[j][0], v.light_intensity[j][1], v.light_intensity[j][2]});
  }
  c.eye = {v.eye[0], v.eye[1], v.eye[2]};
  V3d tg = {v.target[0], v.target[1], v.target[2]};
  V3d up = {v.up[0], v.up[1], v.up[2]};
  c.fwd = nrm(tg - c.eye);
  c.right = nrm(cross(c.fwd, up));
  c.up = cross(c.right, c.fwd);
  c.th = std::tan((double)v.fov_y_deg * PI / 360.0);
  c.W = v.width; c.H = v.height; c.spp = v.spp;
  c.aspect = (double)v.width / (double)v.height;
  c.off = (uint32_t)v.pixel_offset;
  return c;
}

V3d cam_dir(const Cam& c, double px, double py) {
  double sx = 2.0 * px / c.W - 1.0;
  double sy = 1.0 - 2.0 * py / c.H;
  return nrm(c.fwd + scl(c.right, sx * c.th * c.aspect) + scl(c.up, sy * c.th));
}

// ---------------------------------------------------------------- intersection
// Watertight ray/triangle test (Woop, Benthin, Wald 2013) in double; b1, b2 =
// barycentric weights of p1 and p2 at the hit.
bool tri_hit(const V3d& o, const V3d& d, const V3d& p0, const V3d& p1, const V3d& p2, double& t,
             double* b1 = nullptr, double* b2 = nullptr) {
  double ad[3] = {std::fabs(d.x), std::fabs(d.y), std::fabs(d.z)};
  int kz = (ad[0] > ad[1]) ? (ad[0] > ad[2] ? 0 : 2) : (ad[1] > ad[2] ? 1 : 2);
  int kx = (kz + 1) % 3, ky = (kx + 1) % 3;
  if (comp(d, kz) < 0) std::swap(kx, ky);
  double sz = 1.0 / comp(d, kz);
  double sx = comp(d, kx) * sz, sy = comp(d, ky) * sz;
  V3d A = p0 - o, B = p1 - o, C = p2 - o;
  double Ax = comp(A, kx) - sx * comp(A, kz), Ay = comp(A, ky) - sy * comp(A, kz);
  double Bx = comp(B, kx) - sx * comp(B, kz), By = comp(B, ky) - sy * comp(B, kz);
  double Cx = comp(C, kx) - sx * comp(C, kz), Cy = comp(C, ky) - sy * comp(C, kz);
  double U = Cx * By - Cy * Bx, Vb = Ax * Cy - Ay * Cx, W = Bx * Ay - By * Ax;
  if ((U < 0 || Vb < 0 || W < 0) && (U > 0 || Vb > 0 || W > 0)) return false;
  double det = U + Vb + W;
  if (det == 0.0) return false;
  double Az = sz * comp(A, kz), Bz = sz * comp(B, kz), Cz = sz * comp(C, kz);
  double T = U * Az + Vb * Bz + W * Cz;
  t = T / det;
  if (b1) *b1 = Vb / det;
  if (b2) *b2 = W / det;
  return true;
}

struct Hit { int tri; double t, b1, b2; };

Hit closest(const Scene& s, const V3d& o, const V3d& d, int exclude, double tmax, int exclude2 = -1) {
  Hit h{-1, tmax, 0, 0};
  for (int f = 0; f < s.nf; ++f) {
    if (f == exclude || f == exclude2) continue;
    double t, b1, b2;
    const int* fi = &s.face[3 * f];
    if (!tri_hit(o, d, s.vert[fi[0]], s.vert[fi[1]], s.vert[fi[2]], t, &b1, &b2)) continue;
    if (!(t > T_EPS && t < tmax)) continue;
    if (t < h.t || (t == h.t && f < h.tri)) { h.t = t; h.tri = f; h.b1 = b1; h.b2 = b2; }
  }
  return h;
}

bool occluded(const Scene& s, const V3d& o, const V3d& d, int exclude, double tmax) {
  for (int f = 0; f < s.nf; ++f) {
    if (f == exclude) continue;
    double t;
    const int* fi = &s.face[3 * f];
    if (tri_hit(o, d, s.vert[fi[0]], s.vert[fi[1]], s.vert[fi[2]], t) && t > T_EPS && t < tmax)
      return true;
  }
  return false;
}

// ---------------------------------------------------------------- environment
double lum(const double* c) { return 0.2126 * c[0] + 0.7152 * c[1] + 0.0722 * c[2]; }

int build_alias(const float* rgb, int w, int h, std::vector<double>& prob, std::vector<int>& alias,
                std::vector<double>& pmf) {
  // Vose's alias method over texel weights lum * sin(theta at the row centre).
  int N = w * h;
  std::vector<double> wt(N);
  double tot = 0;
  for (int r = 0; r < h; ++r) {
    double st = std::sin(PI * (r + 0.5) / h);
    for (int c = 0; c < w; ++c) {
      const float* p = rgb + 3 * ((size_t)r * w + c);
      double cc[3] = {p[0], p[1], p[2]};
      wt[(size_t)r * w + c] = lum(cc) * st;
    }
  }
  for (int i = 0; i < N; ++i) {
    if (!(wt[i] >= 0)) return 1;
    tot += wt[i];
  }
  if (!(tot > 0)) return 1;
  prob.assign(N, 1.0); alias.resize(N); pmf.resize(N);
  std::vector<double> q(N);
  std::vector<int> small, large;
  for (int i = 0; i < N; ++i) {
    q[i] = (wt[i] * N) / tot;
    pmf[i] = wt[i] / tot;
    alias[i] = i;
    if (q[i] < 1.0) small.push_back(i); else large.push_back(i);
  }
  while (!small.empty() && !large.empty()) {
    int sidx = small.back(); small.pop_back();
    int l = large.back();
    prob[sidx] = q[sidx];
    alias[sidx] = l;
    q[l] = (q[l] + q[sidx]) - 1.0;
    if (q[l] < 1.0) { large.pop_back(); small.push_back(l); }
  }
  for (int i : large) { prob[i] = 1.0; alias[i] = i; }
  for (int i : small) { prob[i] = 1.0; alias[i] = i; }
  return 0;
}

int alias_pick(const double* prob, const int* alias, int N, uint32_t u0, uint32_t u1) {
  int bin = (int)(((uint64_t)(u0 >> 8) * (uint64_t)N) >> 24);
  // The acceptance threshold is the table value rounded to single precision.
  double thr = (double)(float)prob[bin];
  return unif(u1) < thr ? bin : alias[bin];
}

int env_texel(const Scene& s, const V3d& d, double& sin_t) {
  double phi = std::atan2(d.x, -d.z) + PI;
  int col = (int)(phi / (2 * PI) * s.ew);
  col = std::min(std::max(col, 0), s.ew - 1);
  double ct = std::min(std::max(d.y, -1.0), 1.0);
  double th = std::acos(ct);
  int row = (int)(th / PI * s.eh);
  row = std::min(std::max(row, 0), s.eh - 1);
  sin_t = std::sqrt(std::max(0.0, 1.0 - d.y * d.y));
  return row * s.ew + col;
}

double env_pdf(const Scene& s, int texel, double sin_t) {
  if (!(sin_t > 0)) return 0.0;
  double N = (double)s.ew * s.eh;
  return s.pmf[texel] * N / (2.0 * PI * PI * sin_t);
}

// ---------------------------------------------------------------- BRDF
struct Mat { double kd[3], ks[3], alpha; };

template <class T> struct MatT { T kd[3], ks[3], alpha; };

// probability of the specular lobe: mean specular over mean specular + mean diffuse
double lobe_prob(const Mat& m) {
  double ks = (m.ks[0] + m.ks[1] + m.ks[2]) / 3.0;
  double den = ks + (m.kd[0] + m.kd[1] + m.kd[2]) / 3.0;
  if (!(den > 0)) return 0.5;
  return std::min(std::max(ks / den, 0.05), 0.95);
}

template <class T> T clamp_alpha(const T& a) {
  if (vv(a) < 0.01) return T(0.01);
  if (vv(a) > 1.0) return T(1.0);
  return a;
}

template <class T> T D_fn(int brdf, const T& c, const T& a) {
  if (brdf == 0) {
    T a2 = a * a;
    T k = c * c * (a2 - 1.0) + 1.0;
    return a2 / (PI * k * k);
  }
  T c2 = c * c;
  T tan2 = (1.0 - c2) / c2;
  return exp(-tan2 / (a * a)) / (PI * a * a * c2 * c2);
}

template <class T> T G1_fn(int brdf, const T& c, const T& a) {
  if (brdf == 0) {
    T a2 = a * a;
    T q = sqrt(a2 + (1.0 - a2) * c * c);
    return 2.0 * c / (c + q);
  }
  T s2 = 1.0 - c * c;
  if (!(vv(s2) > 0)) return T(1.0);
  T x = c / (a * sqrt(s2));
  return 2.0 / (1.0 + erf(x) + exp(-x * x) / (x * std::sqrt(PI)));
}

// Fresnel factor of the specular lobe at cos(theta_d) = wi . h: held at its
// normal-incidence value ks (fresnel = 0), or Schlick's approximation with
// F0 = ks (fresnel = 1): ks + (1 - ks) (1 - cos theta_d)^5, which reaches 1 at
// grazing and equals ks where wi = wo = h.
template <class T> T fresnel_fn(int fresnel, const T& ks, const T& cih) {
  if (fresnel == 0) return ks;
  T x = 1.0 - cih;
  T x2 = x * x;
  return ks + (1.0 - ks) * (x2 * x2 * x);
}

// f(wi, wo) for unit n, wi, wo; zero unless both cosines are positive.
template <class T>
void brdf_eval(int brdf, int fresnel, const MatT<T>& m, const V3<T>& n, const V3<T>& wi, const V3<T>& wo, T f[3]) {
  T ci = dot(n, wi), co = dot(n, wo);
  if (!(vv(ci) > 0) || !(vv(co) > 0)) { f[0] = f[1] = f[2] = T(0.0); return; }
  V3<T> h = nrm(wi + wo);
  T ch = dot(n, h), cih = dot(wi, h);
  T a = clamp_alpha(m.alpha);
  T spec = D_fn(brdf, ch, a) * G1_fn(brdf, ci, a) * G1_fn(brdf, co, a) / (4.0 * ci * co);
  for (int c = 0; c < 3; ++c) f[c] = m.kd[c] / PI + fresnel_fn(fresnel, m.ks[c], cih) * spec;
}

double brdf_pdf(int brdf, const Mat& m, const V3d& n, const V3d& wi, const V3d& wo) {
  double ci = dot(n, wi), co = dot(n, wo);
  if (!(ci > 0) || !(co > 0)) return 0.0;
  V3d h = nrm(wi + wo);
  double ch = dot(n, h), woh = std::fabs(dot(wo, h));
  double a = clamp_alpha(m.alpha);
  double ps = lobe_prob(m);
  double pd = ci / PI;
  double pspec = D_fn(brdf, ch, a) * ch / (4.0 * woh);
  return (1.0 - ps) * pd + ps * pspec;
}

void onb(const V3d& n, V3d& t, V3d& b) {
  // Helper axis h = (7, 9, 11)/16: exact in binary and on no coordinate axis or
  // plane. The frame is continuous in n except near n = +-h (then a second
  // helper). A frame that switches on the sign of a coordinate of n jumps
  // across a whole great circle, where a symmetric mesh's normals lie exactly
  // and rounding alone would pick the side.
  V3d c = cross(V3d{0.4375, 0.5625, 0.6875}, n);
  double l = len(c);
  if (!(l > 1e-6)) {
    c = cross(V3d{0.6875, -0.4375, 0.5625}, n);
    l = len(c);
  }
  t = scl(c, 1.0 / l);
  b = cross(n, t);
}

void concentric(double u1, double u2, double& x, double& y) {
  // Shirley & Chiu 1997 square-to-disk map.
  double a = 2 * u1 - 1, b = 2 * u2 - 1;
  if (a == 0 && b == 0) { x = y = 0; return; }
  double r, ph;
  if (std::fabs(a) > std::fabs(b)) { r = a; ph = (PI / 4) * (b / a); }
  else { r = b; ph = PI / 2 - (PI / 4) * (a / b); }
  x = r * std::cos(ph); y = r * std::sin(ph);
}

// Returns the mixture pdf of the sampled direction, 0 if the sample is invalid.
double brdf_sample(int brdf, const Mat& m, const V3d& n, const V3d& wo, double ul, double u1, double u2,
                   V3d& wi, int* lobe) {
  V3d t, b;
  onb(n, t, b);
  double ps = lobe_prob(m);
  if (ul < ps) {
    double a = clamp_alpha(m.alpha), a2 = a * a;
    double tan2 = brdf == 0 ? a2 * u1 / (1.0 - u1) : -a2 * std::log(1.0 - u1);
    double ch = 1.0 / std::sqrt(1.0 + tan2);
    double sh = std::sqrt(std::max(0.0, 1.0 - ch * ch));
    double ph = 2 * PI * u2;
    V3d h = scl(t, sh * std::cos(ph)) + scl(b, sh * std::sin(ph)) + scl(n, ch);
    wi = scl(h, 2.0 * dot(wo, h)) - wo;
    if (lobe) *lobe = 1;
  } else {
    double x, y;
    concentric(u1, u2, x, y);
    double z = std::sqrt(std::max(0.0, 1.0 - x * x - y * y));
    wi = scl(t, x) + scl(b, y) + scl(n, z);
    if (lobe) *lobe = 0;
  }
  if (!(dot(n, wi) > 0)) return 0.0;
  return brdf_pdf(brdf, m, n, wi, wo);
}

// ---------------------------------------------------------------- variables
// Registry of the differentiable inputs one path touches (dual-number dims).
struct Vars {
  std::vector<int> vid;   // vertex ids, 3 dims each
  std::vector<int> vdim;
  std::vector<int> fid;   // face ids, 5 dims each
  std::vector<int> fdim;
  std::vector<int> nvid;  // vertex normals (interpolated shading), 3 dims each; scatter_grad
  std::vector<int> nvdim; // carries their derivative on to the vertices around them
  int nd = 0;
  bool overflow = false;  // a variable found no room in MAXD: the path's gradient is incomplete
};

// set when any path of the current call overflowed its dual dimensions (the
// call then reports an error instead of a partial gradient)
std::atomic<bool> g_dual_overflow{false};

template <class T> struct Access;

template <> struct Access<double> {
  static V3<double> vertex(const Scene& s, Vars*, int v) { return s.vert[v]; }
  static V3<double> vnormal(const Scene&, Vars*, int, const V3d& N) { return N; }
  static MatT<double> params(const Scene& s, Vars*, int f) {
    MatT<double> m;
    const double* q = &s.param[(size_t)s.np * f];
    for (int c = 0; c < 3; ++c) m.kd[c] = q[c];
    for (int c = 0; c < 3; ++c) m.ks[c] = q[s.np == 7 ? 3 + c : 3];
    m.alpha = q[s.np - 1];
    return m;
  }
};

inline Dual unit_dual(double v, int dim) {
  Dual d(v);
  d.n = dim + 1;
  for (int k = 0; k < dim; ++k) d.g[k] = 0;
  d.g[dim] = 1.0;
  return d;
}

template <> struct Access<Dual> {
  static V3<Dual> vertex(const Scene& s, Vars* vars, int v) {
    int base = -1;
    for (size_t i = 0; i < vars->vid.size(); ++i)
      if (vars->vid[i] == v) base = vars->vdim[i];
    const V3d& p = s.vert[v];
    if (base < 0) {
      if (vars->nd + 3 > MAXD) { vars->overflow = true; return lift<Dual>(p); }
      base = vars->nd; vars->nd += 3;
      vars->vid.push_back(v); vars->vdim.push_back(base);
    }
    return {unit_dual(p.x, base), unit_dual(p.y, base + 1), unit_dual(p.z, base + 2)};
  }
  // vertex normal N of vertex v as three variables of its own
  static V3<Dual> vnormal(const Scene&, Vars* vars, int v, const V3d& N) {
    int base = -1;
    for (size_t i = 0; i < vars->nvid.size(); ++i)
      if (vars->nvid[i] == v) base = vars->nvdim[i];
    if (base < 0) {
      if (vars->nd + 3 > MAXD) { vars->overflow = true; return lift<Dual>(N); }
      base = vars->nd; vars->nd += 3;
      vars->nvid.push_back(v); vars->nvdim.push_back(base);
    }
    return {unit_dual(N.x, base), unit_dual(N.y, base + 1), unit_dual(N.z, base + 2)};
  }
  static MatT<Dual> params(const Scene& s, Vars* vars, int f) {
    int base = -1;
    for (size_t i = 0; i < vars->fid.size(); ++i)
      if (vars->fid[i] == f) base = vars->fdim[i];
    const double* q = &s.param[(size_t)s.np * f];
    MatT<Dual> m;
    if (base < 0 && vars->nd + s.np > MAXD) {
      vars->overflow = true;
      for (int c = 0; c < 3; ++c) m.kd[c] = Dual(q[c]);
      for (int c = 0; c < 3; ++c) m.ks[c] = Dual(q[s.np == 7 ? 3 + c : 3]);
      m.alpha = Dual(q[s.np - 1]);
      return m;
    }
    if (base < 0) {
      base = vars->nd; vars->nd += s.np;
      vars->fid.push_back(f); vars->fdim.push_back(base);
    }
    for (int c = 0; c < 3; ++c) m.kd[c] = unit_dual(q[c], base + c);
    // one specular value for all channels (5 parameters) or one per channel (7)
    for (int c = 0; c < 3; ++c) m.ks[c] = s.np == 7 ? unit_dual(q[3 + c], base + 3 + c) : unit_dual(q[3], base + 3);
    m.alpha = unit_dual(q[s.np - 1], base + s.np - 1);
    return m;
  }
};

// Mesh-colors texel of the hit (Sec. 3.3): k = (t (r+1)(r+2) + i (2r - i + 3)) / 2 + j,
// (i, j) = floor(r (alpha, beta)), alpha and beta the barycentric weights of the
// face's second and third vertices; clamped so rounding cannot leave the face's block.
long long texel(const Scene& s, int t, double alpha, double beta) {
  if (s.res == 0) return t;
  long long r = s.res;
  long long i = std::min<long long>(std::max<long long>((long long)std::floor(r * alpha), 0), r);
  long long j = std::min<long long>(std::max<long long>((long long)std::floor(r * beta), 0), r - i);
  return (t * (r + 1) * (r + 2) + i * (2 * r - i + 3)) / 2 + j;
}

Mat mat_val(const Scene& s, int f) {
  Mat m;
  const double* q = &s.param[(size_t)s.np * f];
  for (int c = 0; c < 3; ++c) m.kd[c] = q[c];
  for (int c = 0; c < 3; ++c) m.ks[c] = q[s.np == 7 ? 3 + c : 3];
  m.alpha = q[s.np - 1];
  return m;
}

// ---------------------------------------------------------------- tape
// Record/replay of every quantity the gradient treats as constant (sampled
// directions, pdfs, MIS weights, the sampled texel). Replaying a recorded tape
// under perturbed inputs evaluates the estimator with sampling detached, which
// is what finite differences must use to check the dual-number gradient.
struct Tape {
  int mode = 0;  // 0 off, 1 record, 2 replay
  std::vector<double> v;
  size_t pos = 0;
  bool bad = false;
  double take(double x) {
    if (mode == 1) v.push_back(x);
    else if (mode == 2) { if (pos < v.size()) x = v[pos++]; else bad = true; }
    return x;
  }
  V3d take(const V3d& a) { return V3d{take(a.x), take(a.y), take(a.z)}; }
};

// ---------------------------------------------------------------- edges
struct Edge { int a, b; int f[2]; int nf; };

std::vector<Edge> edge_list(const Scene& s) {
  std::map<std::pair<int, int>, Edge> m;
  for (int f = 0; f < s.nf; ++f)
    for (int k = 0; k < 3; ++k) {
      int a = s.face[3 * f + k], b = s.face[3 * f + (k + 1) % 3];
      std::pair<int, int> key(std::min(a, b), std::max(a, b));
      auto it = m.find(key);
      if (it == m.end()) {
        Edge e{key.first, key.second, {f, -1}, 1};
        m.emplace(key, e);
      } else {
        if (it->second.nf < 2) it->second.f[it->second.nf] = f;
        it->second.nf++;
      }
    }
  std::vector<Edge> out;
  out.reserve(m.size());
  for (auto& kv : m) out.push_back(kv.second);  // std::map iterates in (min, max) order
  return out;
}

// Secondary-visibility edge sampling context: the mesh's edge list and the
// candidate rule (0 = silhouettes as seen from the vertex, 1 = every edge).
// Hierarchy over the edges for the importance-sampled secondary edge pick:
// leaves are blocks of G consecutive edges in edge order (at most 2^14 blocks),
// a complete binary tree above them in heap order (root 1, leaf i at 2^L + i);
// each node keeps the box of its edges' endpoints and their summed length.
struct EdgeTree {
  int G = 4, L = 0, nleaf = 0, nE = 0;
  std::vector<V3d> lo, hi;
  std::vector<double> S;
  // cone of the unit normals of the faces on the node's edges: axis, cos of the
  // half-angle; cos < -1.5 marks a node whose silhouettes cannot be bounded (an
  // edge with one face or more than two, or normals spread too wide)
  std::vector<V3d> ax;
  std::vector<double> ct;
  std::vector<char> any;   // the node holds an edge of nonzero length
};

double angle_of(double c) { return std::acos(std::max(-1.0, std::min(1.0, c))); }

EdgeTree edge_tree(const Scene& s, const std::vector<Edge>& E) {
  EdgeTree t;
  t.nE = (int)E.size();
  t.G = std::max(4, (t.nE + (1 << 14) - 1) >> 14);
  t.nleaf = (t.nE + t.G - 1) / t.G;
  while ((1 << t.L) < t.nleaf) ++t.L;
  size_t nn = (size_t)2 << t.L;
  t.lo.assign(nn, V3d{INFINITY, INFINITY, INFINITY});
  t.hi.assign(nn, V3d{-INFINITY, -INFINITY, -INFINITY});
  t.S.assign(nn, 0.0);
  t.ax.assign(nn, V3d{0, 0, 0});
  t.ct.assign(nn, -2.0);
  t.any.assign(nn, 0);
  auto unit_normal = [&](int f) {
    const int* fi = &s.face[3 * f];
    return nrm(cross(s.vert[fi[1]] - s.vert[fi[0]], s.vert[fi[2]] - s.vert[fi[0]]));
  };
  auto grow = [&](size_t k, const V3d& a) {
    t.lo[k] = {std::min(t.lo[k].x, a.x), std::min(t.lo[k].y, a.y), std::min(t.lo[k].z, a.z)};
    t.hi[k] = {std::max(t.hi[k].x, a.x), std::max(t.hi[k].y, a.y), std::max(t.hi[k].z, a.z)};
  };
  for (int i = 0; i < t.nleaf; ++i) {
    size_t k = ((size_t)1 << t.L) + i;
    bool bounded = true;
    V3d sum{0, 0, 0};
    for (int e = i * t.G; e < std::min(t.nE, (i + 1) * t.G); ++e) {
      const V3d &A = s.vert[E[e].a], &B = s.vert[E[e].b];
      grow(k, A);
      grow(k, B);
      double l = len(B - A);
      t.S[k] += l;
      if (l > 0) t.any[k] = 1;
      if (E[e].nf != 2) { bounded = false; continue; }
      sum = sum + unit_normal(E[e].f[0]) + unit_normal(E[e].f[1]);
    }
    double sl = len(sum);
    if (!t.any[k] || !bounded || !(sl > 1e-6)) continue;
    t.ax[k] = scl(sum, 1.0 / sl);
    double c = 1.0;
    for (int e = i * t.G; e < std::min(t.nE, (i + 1) * t.G); ++e)
      c = std::min(c, std::min(dot(t.ax[k], unit_normal(E[e].f[0])), dot(t.ax[k], unit_normal(E[e].f[1]))));
    t.ct[k] = c > 0.0 ? c : -2.0;    // cones wider than a hemisphere bound nothing
  }
  for (size_t k = ((size_t)1 << t.L) - 1; k >= 1; --k) {
    const V3d &la = t.lo[2 * k], &lb = t.lo[2 * k + 1], &ha = t.hi[2 * k], &hb = t.hi[2 * k + 1];
    t.lo[k] = {std::min(la.x, lb.x), std::min(la.y, lb.y), std::min(la.z, lb.z)};
    t.hi[k] = {std::max(ha.x, hb.x), std::max(ha.y, hb.y), std::max(ha.z, hb.z)};
    t.S[k] = t.S[2 * k] + t.S[2 * k + 1];
    // the cone around the normalised sum of the children's axes that holds both
    size_t a = 2 * k, b = 2 * k + 1;
    t.any[k] = t.any[a] | t.any[b];
    if (!t.any[a] || !t.any[b]) {
      size_t o = t.any[a] ? a : b;
      t.ax[k] = t.ax[o];
      t.ct[k] = t.ct[o];
      continue;
    }
    if (t.ct[a] < -1.5 || t.ct[b] < -1.5) continue;
    V3d sum = t.ax[a] + t.ax[b];
    double sl = len(sum);
    if (!(sl > 1e-6)) continue;
    t.ax[k] = scl(sum, 1.0 / sl);
    double th = std::max(angle_of(dot(t.ax[k], t.ax[a])) + angle_of(t.ct[a]),
                         angle_of(dot(t.ax[k], t.ax[b])) + angle_of(t.ct[b]));
    t.ct[k] = th < 0.5 * PI ? std::cos(th) : -2.0;
  }
  return t;
}

// Importance of node k at a path vertex (p, tangent plane normal n, band bnd):
// 0 when the whole box lies at or below the plane (no edge in it can be
// sampled) or, for silhouette sampling (sil), when every face on the node's
// edges sees p on the same side (no edge in it is a silhouette from p); else
// the summed length over max(d^2, diag^2 / 4), d the distance from p to the box.
// Side bound: n_f.(p - x) for x in the box and n_f in the cone (axis a, half-
// angle th) lies within |v| cos(phi -+ th) -+ r, v = p - c, c the box centre, r
// its half-diagonal, phi the angle between a and v.
double tree_weight(const EdgeTree& t, size_t k, const V3d& p, const V3d& n, double bnd, bool sil) {
  if (!(t.S[k] > 0)) return 0.0;
  const V3d &lo = t.lo[k], &hi = t.hi[k];
  double top = (n.x > 0 ? hi.x - p.x : lo.x - p.x) * n.x + (n.y > 0 ? hi.y - p.y : lo.y - p.y) * n.y +
               (n.z > 0 ? hi.z - p.z : lo.z - p.z) * n.z;
  if (!(top > bnd)) return 0.0;
  if (sil && t.ct[k] > -1.5) {
    V3d c = scl(lo + hi, 0.5), v = p - c;
    double r = 0.5 * len(hi - lo), D = len(v);
    if (D > r) {
      double cp = dot(t.ax[k], v) / D, sp = std::sqrt(std::max(0.0, 1.0 - cp * cp));
      double cq = t.ct[k], sq = std::sqrt(std::max(0.0, 1.0 - cq * cq));
      double cmin = cp <= -cq ? -1.0 : cp * cq - sp * sq;
      double cmax = cp >= cq ? 1.0 : cp * cq + sp * sq;
      if (D * cmin - r > -bnd || D * cmax + r < bnd) return 0.0;
    }
  }
  double dx = std::max(lo.x - p.x, std::max(0.0, p.x - hi.x));
  double dy = std::max(lo.y - p.y, std::max(0.0, p.y - hi.y));
  double dz = std::max(lo.z - p.z, std::max(0.0, p.z - hi.z));
  double ex = hi.x - lo.x, ey = hi.y - lo.y, ez = hi.z - lo.z;
  double den = std::max(dx * dx + dy * dy + dz * dz, 0.25 * (ex * ex + ey * ey + ez * ez));
  return t.S[k] / std::max(den, 1e-30);
}

// Descends the tree with one uniform per level (level j: word j % 4 of the
// draw (c0, c1, b<<4 | (4 + j/4), stream)), then picks uniformly in the leaf
// block with the word uleaf. Returns the edge or -1; prob = its probability.
int tree_pick(const EdgeTree& t, const Rng& rng, uint32_t c0, uint32_t c1, int b, uint32_t stream, const V3d& p,
              const V3d& n, double bnd, bool sil, uint32_t uleaf, double& prob) {
  size_t k = 1;
  prob = 1.0;
  U4 u{};
  for (int j = 0; j < t.L; ++j) {
    if (j % 4 == 0) u = rng.draw(c0, c1, (uint32_t)(b << 4) | (4u + (uint32_t)(j / 4)), stream);
    double wa = tree_weight(t, 2 * k, p, n, bnd, sil), wb = tree_weight(t, 2 * k + 1, p, n, bnd, sil);
    if (!(wa + wb > 0)) return -1;
    if (unif(u.w[j % 4]) < wa / (wa + wb)) { k = 2 * k; prob *= wa / (wa + wb); }
    else { k = 2 * k + 1; prob *= wb / (wa + wb); }
  }
  int first = (int)(k - ((size_t)1 << t.L)) * t.G;
  int cnt = std::min(t.G, t.nE - first);
  if (cnt <= 0) return -1;
  prob /= cnt;
  return first + (int)(((uint64_t)(uleaf >> 8) * (uint64_t)cnt) >> 24);
}

// mode: silhouettes or every edge; sampling 1: uniform over all edges, 2: by the tree
struct SecCtx { const std::vector<Edge>* E; int mode; int sampling = 1; const EdgeTree* T = nullptr; };

// Signed distance of p from the plane of face f (unit normal of the face's winding).
double face_side(const Scene& s, int f, const V3d& p) {
  const int* fi = &s.face[3 * f];
  V3d a = s.vert[fi[0]];
  V3d m = nrm(cross(s.vert[fi[1]] - a, s.vert[fi[2]] - a));
  return dot(m, p - a);
}

template <class T>
void trace_path(const Scene& s, const Rng& rng, int B, const Lights& lt, const V3d& eye, const V3d& d0, uint32_t c0,
                uint32_t c1, uint32_t stream, Vars* vars, T L[3], long long& segments, Tape* tape = nullptr,
                const SecCtx* sec = nullptr, int b0 = 0, int origin0 = -1, uint64_t* sig = nullptr);

// One secondary-visibility edge sample at path vertex b (the boundary term of
// the vertex's integral over incoming directions; Li et al.'s edge sampling,
// which the paper's gradient relies on, Sec. 3.2). The integrand g(w) = f cos
// L_in(w) jumps where the direction crosses the image of a mesh edge on the
// vertex's sphere of directions; moving the edge's endpoints (x) or the vertex
// (p) moves that arc by m.(dx - dp)/r along its normal m. The boundary term
// integral over the arc of (g(w - eps m) - g(w + eps m)) m.(dx - dp)/r is
// estimated with one edge picked uniformly from all E mesh edges, one point x
// uniform along the part of it above the vertex's tangent plane, and two side
// paths (shared random numbers, stream 16 + b) that continue the path from
// vertex b + 1. Arc length per unit edge length is |w x t|/r, t the unit edge
// direction, so the sample's weight is |w x t| E len (tau1 - tau0) / r^2 times
// T_b (g- - g+). It is added to L as a dual with zero value whose derivative is
// that weight times m.(dx - dp), dx = (1 - tau) dA + tau dB.
void secondary_edge(const Scene& s, const Rng& rng, int B, const Lights& lt, int b, const V3<Dual>& p, const V3d& nv,
                    const V3d& ns, const V3d& wo,
                    int f0, long long tex, const Dual thr[3], uint32_t c0, uint32_t c1, uint32_t stream,
                    const SecCtx& sc, Vars* vars, Dual L[3], long long& segments) {
  const std::vector<Edge>& E = *sc.E;
  if (E.empty()) return;
  U4 u = rng.draw(c0, c1, (uint32_t)(b << 4) | 3u, stream);
  uint64_t nE = E.size();
  V3d pv = val(p);
  double bnd = SEC_BAND * (1.0 + std::max(std::fabs(pv.x), std::max(std::fabs(pv.y), std::fabs(pv.z))));
  size_t ei;
  double inv_p;   // 1 / pick probability
  if (sc.sampling == 2) {
    double pr;
    int k = tree_pick(*sc.T, rng, c0, c1, b, stream, pv, nv, bnd, sc.mode == 0, u.w[0], pr);
    if (k < 0) return;
    ei = (size_t)k;
    inv_p = 1.0 / pr;
  } else {
    ei = (size_t)(((uint64_t)(u.w[0] >> 8) * nE) >> 24);
    inv_p = (double)nE;
  }
  const Edge& e = E[ei];
  if (e.f[0] == f0 || (e.nf == 2 && e.f[1] == f0)) return;   // its arc lies on the vertex's horizon
  V3d A = s.vert[e.a], Bv = s.vert[e.b];
  if (sc.mode == 0) {
    double s1 = face_side(s, e.f[0], pv);
    bool sil;
    if (e.nf == 2) {
      double s2 = face_side(s, e.f[1], pv);
      sil = (s1 > bnd && s2 < -bnd) || (s1 < -bnd && s2 > bnd);
    } else {
      sil = std::fabs(s1) > bnd;
    }
    if (!sil) return;
  }
  // the part of the edge above the tangent plane (below it the BRDF is zero);
  // with shading normals, above the shading plane as well
  double t0 = 0.0, t1 = 1.0;
  for (int pl = 0; pl < (s.smooth ? 2 : 1); ++pl) {
    const V3d& nc = pl == 0 ? nv : ns;
    double hA = dot(nc, A - pv), hB = dot(nc, Bv - pv);
    if (!(hA > bnd) && !(hB > bnd)) return;
    if (!(hA > bnd)) t0 = std::max(t0, (bnd - hA) / (hB - hA));
    if (!(hB > bnd)) t1 = std::min(t1, (hA - bnd) / (hA - hB));
  }
  if (!(t1 > t0)) return;
  double tau = t0 + unif(u.w[1]) * (t1 - t0);
  V3d tv = Bv - A;
  V3d x = A + scl(tv, tau);
  V3d dv = x - pv;
  double r = len(dv);
  if (!(r > SEC_RMIN)) return;
  V3d w = scl(dv, 1.0 / r);
  double l = len(tv);
  V3d cr = cross(w, scl(tv, 1.0 / l));
  double sn = len(cr);
  if (!(sn > SEC_SMIN)) return;
  V3d mh = scl(cr, 1.0 / sn);
  double coef = sn * inv_p * l * (t1 - t0) / (r * r);
  MatT<double> m = Access<double>::params(s, nullptr, (int)tex);
  double g[2][3];
  for (int side = 0; side < 2; ++side) {
    V3d ws = nrm(w + scl(mh, side == 0 ? -SEC_EPS : SEC_EPS));
    double f[3], Li[3];
    brdf_eval(s.brdf, s.fresnel, m, ns, ws, wo, f);
    double ci = dot(ns, ws);
    if (s.smooth && !(dot(nv, ws) > 0)) ci = 0;
    trace_path<double>(s, rng, B, lt, pv, ws, c0, c1, 16u + (uint32_t)b, nullptr, Li, segments, nullptr, nullptr, b + 1,
                       f0);
    for (int c = 0; c < 3; ++c) g[side][c] = ci > 0 ? f[c] * ci * Li[c] : 0.0;
  }
  double k[3];
  bool any = false;
  for (int c = 0; c < 3; ++c) {
    k[c] = thr[c].v * (g[0][c] - g[1][c]) * coef;
    any |= k[c] != 0.0;
  }
  if (!any) return;
  V3<Dual> Ad = Access<Dual>::vertex(s, vars, e.a), Bd = Access<Dual>::vertex(s, vars, e.b);
  V3<Dual> xd = scl(Ad, 1.0 - tau) + scl(Bd, tau);
  Dual ed = dot(lift<Dual>(mh), xd - p);
  Dual z = ed - ed.v;
  for (int c = 0; c < 3; ++c) L[c] = L[c] + z * k[c];
}

// ---------------------------------------------------------------- shading normals
// Interpolated shading normals (scene option; the paper's facets are flat, the
// variant is a standard one). Vertex normal N_v = M_v / |M_v|, M_v = the sum of
// e1 x e2 = (v1 - v0) x (v2 - v0) over the faces around v (area weighting), in
// face order. At a hit p on face (v0, v1, v2) with m = e1 x e2 the barycentric
// weights are b1 = ((p - v0) x e2).m / m.m and b2 = (e1 x (p - v0)).m / m.m (p
// on the face's plane), and n_s = s / |s|, s = (1 - b1 - b2) N0 + b1 N1 + b2 N2,
// turned with the geometric normal toward the incoming direction. Everything is
// differentiated: each vertex normal is a variable of the path, and its
// derivative goes on to the vertices of the faces around the vertex
// (vertex_normal_chain), so a path's variables do not grow with the valence.
V3d vertex_normal_value(const Scene& s, int v, double* mlen = nullptr) {
  V3d M{0, 0, 0};
  for (int k = s.vf_start[v]; k < s.vf_start[(size_t)v + 1]; ++k) {
    const int* fi = &s.face[3 * (size_t)s.vf_list[k]];
    M = M + cross(s.vert[fi[1]] - s.vert[fi[0]], s.vert[fi[2]] - s.vert[fi[0]]);
  }
  if (mlen) *mlen = len(M);
  return nrm(M);
}

template <class T>
V3<T> vertex_normal_of(const Scene& s, Vars* vars, int v) {
  return Access<T>::vnormal(s, vars, v, vertex_normal_value(s, v));
}

// d/dN of vertex v's normal to the vertices: N = M / |M| gives dM = (dN - N
// (N.dN)) / |M|; each face's (v1 - v0) x (v2 - v0), a term of M, passes dM on
// as v1: e2 x dM, v2: dM x e1, v0: minus both.
void vertex_normal_chain(const Scene& s, int v, const V3d& gN, double* dv) {
  double ml;
  V3d N = vertex_normal_value(s, v, &ml);
  if (!(ml > 0)) return;
  V3d gM = scl(gN - scl(N, dot(N, gN)), 1.0 / ml);
  for (int k = s.vf_start[v]; k < s.vf_start[(size_t)v + 1]; ++k) {
    const int* fi = &s.face[3 * (size_t)s.vf_list[k]];
    V3d e1 = s.vert[fi[1]] - s.vert[fi[0]], e2 = s.vert[fi[2]] - s.vert[fi[0]];
    V3d g1 = cross(e2, gM), g2 = cross(gM, e1);
    V3d g0 = -(g1 + g2);
    const V3d* g[3] = {&g0, &g1, &g2};
    for (int j = 0; j < 3; ++j) {
      dv[3 * fi[j]] += g[j]->x; dv[3 * fi[j] + 1] += g[j]->y; dv[3 * fi[j] + 2] += g[j]->z;
    }
  }
}

// shading normal at p of face fi (vertices v0, v1, v2, m = e1 x e2), sign = +1 or
// -1 as the geometric normal was turned
template <class T>
V3<T> shading_normal(const Scene& s, Vars* vars, const int* fi, const V3<T>& v0, const V3<T>& v1, const V3<T>& v2,
                     const V3<T>& m, const V3<T>& p, double sign) {
  V3<T> e1 = v1 - v0, e2 = v2 - v0, q = p - v0;
  T mm = dot(m, m);
  T b1 = dot(cross(q, e2), m) / mm;
  T b2 = dot(cross(e1, q), m) / mm;
  V3<T> N0 = vertex_normal_of<T>(s, vars, fi[0]), N1 = vertex_normal_of<T>(s, vars, fi[1]),
        N2 = vertex_normal_of<T>(s, vars, fi[2]);
  V3<T> sv = scl(N0, 1.0 - b1 - b2) + scl(N1, b1) + scl(N2, b2);
  return scl(nrm(sv), sign);
}

// ---------------------------------------------------------------- one path
// Radiance of one path whose primary ray is (eye, d0). Counter words (c0, c1,
// stream) identify the path; `segments` counts ray queries.
// b0 > 0 starts a path at vertex b0 from a point on face origin0 (a side path of
// a secondary edge sample): its first ray collects the environment unweighted,
// and a first ray that would find vertex B adds nothing.
template <class T>
void trace_path(const Scene& s, const Rng& rng, int B, const Lights& lt, const V3d& eye, const V3d& d0, uint32_t c0,
                uint32_t c1, uint32_t stream, Vars* vars, T L[3], long long& segments, Tape* tape,
                const SecCtx* sec, int b0, int origin0, uint64_t* sig) {
  using A = Access<T>;
  uint64_t hsig = SIG_BASIS;
  auto mix = [&](uint32_t x) { hsig = sig_mix(hsig, x); };
  struct SigOut {
    uint64_t* out; const uint64_t* h;
    ~SigOut() { if (out) *out = *h; }
  } sig_out{sig, &hsig};
  Tape none;
  Tape& tp = tape ? *tape : none;
  for (int c = 0; c < 3; ++c) L[c] = T(0.0);
  T thr[3] = {T(1.0), T(1.0), T(1.0)};
  V3<T> o = lift<T>(eye);
  V3d d = d0;
  int origin = origin0;
  double last_pdf = 0;
  for (int b = b0;; ++b) {
    ++segments;
    Hit h = closest(s, val(o), d, origin, INFINITY);
    if (h.tri < 0) mix(0xffffffffu);
    else if (b < B) mix((uint32_t)h.tri);
    if (h.tri < 0) {
      if (s.ew > 0) {
        double st;
        int tx = env_texel(s, d, st);
        mix((uint32_t)tx);   // the nearest-texel lookup is a decision too
        double w = 1.0;
        if (b > b0) {
          double pe = env_pdf(s, tx, st);
          w = last_pdf * last_pdf / (last_pdf * last_pdf + pe * pe);
        }
        w = tp.take(w);
        for (int c = 0; c < 3; ++c) L[c] = L[c] + thr[c] * (s.env[3 * tx + c] * w);
      }
      return;
    }
    if (b >= B) return;
    const int* fi = &s.face[3 * h.tri];
    V3<T> v0 = A::vertex(s, vars, fi[0]);
    V3<T> v1 = A::vertex(s, vars, fi[1]);
    V3<T> v2 = A::vertex(s, vars, fi[2]);
    long long tex = texel(s, h.tri, h.b1, h.b2);
    if (s.res > 0) mix((uint32_t)tex);   // so is the mesh-colors texel of the hit
    MatT<T> m = A::params(s, vars, (int)tex);
    Mat mv = mat_val(s, (int)tex);
    V3<T> mvec = cross(v1 - v0, v2 - v0);
    V3<T> dT = lift<T>(d);
    T t = dot(v0 - o, mvec) / dot(dT, mvec);
    V3<T> p = o + scl(dT, t);
    V3<T> ng = nrm(mvec);
    V3d wo_d = -d;
    V3<T> wo = lift<T>(wo_d);
    V3<T> n = (dot(val(ng), wo_d) < 0) ? -ng : ng;
    V3d nv = val(n), pv = val(p);
    // shading normal: the geometric one, or interpolated from the vertex normals;
    // a direction counts only above both
    V3<T> ns = s.smooth ? shading_normal<T>(s, vars, fi, v0, v1, v2, mvec, p, dot(val(ng), wo_d) < 0 ? -1.0 : 1.0)
                        : n;
    V3d nsv = val(ns);

    // next-event estimation: point lights
    bool traced = false;      // any shadow ray at this vertex
    uint32_t vis = 0;         // bit j: light j seen; bit 8: the environment sample seen
    for (size_t j = 0; j < lt.pos.size(); ++j) {
      V3<T> dv = lift<T>(lt.pos[j]) - p;
      T dist = len(dv);
      V3<T> wi = scl(dv, 1.0 / dist);
      T ci = dot(ns, wi);
      if (!(vv(dot(n, wi)) > 0) || !(vv(ci) > 0) || !(vv(dist) > 2 * T_EPS)) continue;
      ++segments;
      traced = true;
      if (occluded(s, pv, val(wi), h.tri, vv(dist) - T_EPS)) continue;
      vis |= 1u << j;
      T f[3];
      brdf_eval(s.brdf, s.fresnel, m, ns, wi, wo, f);
      T g = ci / (dist * dist);
      for (int c = 0; c < 3; ++c) L[c] = L[c] + thr[c] * f[c] * g * comp(lt.I[j], c);
    }
    // next-event estimation: environment
    if (s.ew > 0) {
      U4 u = rng.draw(c0, c1, (uint32_t)(b << 4) | 1u, stream);
      int N = s.ew * s.eh;
      int tx = alias_pick(s.prob.data(), s.alias.data(), N, u.w[0], u.w[1]);
      mix((uint32_t)tx);
      int row = tx / s.ew, col = tx % s.ew;
      double uu = (col + unif(u.w[2])) / s.ew, vq = (row + unif(u.w[3])) / s.eh;
      double th = PI * vq, ph = 2 * PI * uu;
      double st = std::sin(th), ct = std::cos(th);
      V3d wi = {-st * std::sin(ph), ct, st * std::cos(ph)};
      tx = (int)tp.take((double)tx);
      st = tp.take(st);
      wi = tp.take(wi);
      if (st > 0) {
        T ci = dot(ns, lift<T>(wi));
        if (vv(dot(n, lift<T>(wi))) > 0 && vv(ci) > 0) {
          ++segments;
          traced = true;
          if (!occluded(s, pv, wi, h.tri, INFINITY)) {
            vis |= 1u << 8;
            double pe = env_pdf(s, tx, st);
            double w = 1.0;
            if (b < B - 1) {
              double pb = brdf_pdf(s.brdf, mv, nsv, wi, wo_d);
              w = pe * pe / (pe * pe + pb * pb);
            }
            pe = tp.take(pe);
            w = tp.take(w);
            T f[3];
            brdf_eval(s.brdf, s.fresnel, m, ns, lift<T>(wi), wo, f);
            for (int c = 0; c < 3; ++c) L[c] = L[c] + thr[c] * f[c] * ci * (s.env[3 * tx + c] * w / pe);
          }
        }
      }
    }
    if constexpr (std::is_same<T, Dual>::value) {
      if (sec)
        secondary_edge(s, rng, B, lt, b, p, nv, nsv, wo_d, h.tri, tex, thr, c0, c1, stream, *sec, vars, L, segments);
    }
    if (b == B - 1) {
      if (traced) mix(vis);
      return;
    }
    // BSDF sampling (direction and pdf held constant under differentiation)
    U4 u = rng.draw(c0, c1, (uint32_t)(b << 4) | 2u, stream);
    V3d wi;
    int lobe = 0;
    double pdf = brdf_sample(s.brdf, mv, nsv, wo_d, unif(u.w[0]), unif(u.w[1]), unif(u.w[2]), wi, &lobe);
    if (s.smooth && pdf > 0 && !(dot(nv, wi) > 0)) pdf = 0;   // below the geometric surface
    mix((uint32_t)lobe | (pdf > 0 ? 2u : 0u));
    if (traced) mix(vis);
    pdf = tp.take(pdf);
    wi = tp.take(wi);
    if (!(pdf > 0)) return;
    T f[3];
    V3<T> wiT = lift<T>(wi);
    brdf_eval(s.brdf, s.fresnel, m, ns, wiT, wo, f);
    T ci = dot(ns, wiT);
    for (int c = 0; c < 3; ++c) thr[c] = thr[c] * f[c] * ci / pdf;
    o = p; d = wi; origin = h.tri; last_pdf = pdf;
  }
}

// ---------------------------------------------------------------- helpers
bool load_scene(const orc_scene* in, Scene& s) {
  if (!in || in->n_vertices <= 0 || in->n_faces <= 0 || !in->vertices || !in->faces || !in->face_params)
    return false;
  s.nv = in->n_vertices; s.nf = in->n_faces; s.brdf = in->brdf;
  s.vert.resize(s.nv);
  for (int i = 0; i < s.nv; ++i) s.vert[i] = {in->vertices[3 * i], in->vertices[3 * i + 1], in->vertices[3 * i + 2]};
  s.face.assign(in->faces, in->faces + 3 * (size_t)s.nf);
  for (int v : s.face) if (v < 0 || v >= s.nv) return false;
  if (in->color_res < 0 || in->color_res > 64) return false;
  s.res = in->color_res;
  s.ntex = (s.res + 1) * (s.res + 2) / 2;
  if (in->param_width != 5 && in->param_width != 7) return false;
  s.np = in->param_width;
  if (in->smooth_normals != 0 && in->smooth_normals != 1) return false;
  s.smooth = in->smooth_normals == 1;
  if (in->fresnel != 0 && in->fresnel != 1) return false;
  s.fresnel = in->fresnel;
  s.vf_start.assign((size_t)s.nv + 1, 0);
  for (int v : s.face) ++s.vf_start[(size_t)v + 1];
  for (int v = 0; v < s.nv; ++v) s.vf_start[(size_t)v + 1] += s.vf_start[v];
  s.vf_list.resize(s.face.size());
  {
    std::vector<int> cur(s.vf_start.begin(), s.vf_start.end() - 1);
    for (int f = 0; f < s.nf; ++f)
      for (int k = 0; k < 3; ++k) s.vf_list[(size_t)cur[s.face[3 * f + k]]++] = f;
  }
  s.param.resize((size_t)s.np * s.nf * s.ntex);
  for (size_t i = 0; i < s.param.size(); ++i) s.param[i] = in->face_params[i];
  for (int j = 0; j < in->n_lights; ++j) {
    s.lpos.push_back({in->light_pos[3 * j], in->light_pos[3 * j + 1], in->light_pos[3 * j + 2]});
    s.lint.push_back({in->light_intensity[3 * j], in->light_intensity[3 * j + 1], in->light_intensity[3 * j + 2]});
  }
  if (in->env_width > 0 && in->env_height > 0 && in->env_rgb) {
    s.ew = in->env_width; s.eh = in->env_height;
    s.env.resize(3 * (size_t)s.ew * s.eh);
    for (size_t i = 0; i < s.env.size(); ++i) s.env[i] = in->env_rgb[i];
    if (build_alias(in->env_rgb, s.ew, s.eh, s.prob, s.alias, s.pmf)) return false;
  }
  return true;
}

int nthreads(const orc_params* p) {
  int n = p && p->n_threads > 0 ? p->n_threads : (int)std::thread::hardware_concurrency();
  return std::max(1, n);
}

template <class F> void parallel_for(int n, int nt, F fn) {
  nt = std::max(1, std::min(nt, n));
  std::vector<std::thread> th;
  for (int t = 0; t < nt; ++t)
    th.emplace_back([=]() { for (int i = t; i < n; i += nt) fn(t, i); });
  for (auto& x : th) x.join();
}

void scatter_grad(const Scene& s, const Vars& vars, const Dual& loss, double* dv, double* df, int np) {
  if (vars.overflow) g_dual_overflow = true;
  for (size_t i = 0; i < vars.nvid.size(); ++i) {
    int d = vars.nvdim[i];
    V3d gN{d < loss.n ? loss.g[d] : 0.0, d + 1 < loss.n ? loss.g[d + 1] : 0.0, d + 2 < loss.n ? loss.g[d + 2] : 0.0};
    vertex_normal_chain(s, vars.nvid[i], gN, dv);
  }
  for (size_t i = 0; i < vars.vid.size(); ++i)
    for (int k = 0; k < 3; ++k) {
      int dim = vars.vdim[i] + k;
      if (dim < loss.n) dv[3 * vars.vid[i] + k] += loss.g[dim];
    }
  for (size_t i = 0; i < vars.fid.size(); ++i)
    for (int k = 0; k < np; ++k) {
      int dim = vars.fdim[i] + k;
      if (dim < loss.n && df) df[(size_t)np * vars.fid[i] + k] += loss.g[dim];
    }
}

struct Cand { int e; double t0, t1, len; V3d sa, sb; };

bool project(const Cam& c, const V3d& X, double& px, double& py) {
  V3d rel = X - c.eye;
  double z = dot(rel, c.fwd);
  if (!(z > Z_NEAR)) return false;
  double sx = dot(rel, c.right) / (z * c.th * c.aspect);
  double sy = dot(rel, c.up) / (z * c.th);
  px = (sx + 1.0) * c.W / 2.0;
  py = (1.0 - sy) * c.H / 2.0;
  return true;
}

// derivative of the pixel coordinates of X along screen direction (nx, ny)
V3d proj_jt(const Cam& c, const V3d& X, double nx, double ny) {
  V3d rel = X - c.eye;
  double z = dot(rel, c.fwd);
  double k = c.th * c.aspect;
  double sx = dot(rel, c.right) / (z * k);
  double sy = dot(rel, c.up) / (z * c.th);
  V3d dpx = scl(c.right - scl(c.fwd, sx * k), (c.W / 2.0) / (z * k));
  V3d dpy = scl(c.up - scl(c.fwd, sy * c.th), -(c.H / 2.0) / (z * c.th));
  return scl(dpx, nx) + scl(dpy, ny);
}

bool facing(const Scene& s, int f, const V3d& eye) {
  const int* fi = &s.face[3 * f];
  V3d m = cross(s.vert[fi[1]] - s.vert[fi[0]], s.vert[fi[2]] - s.vert[fi[0]]);
  return dot(m, eye - s.vert[fi[0]]) > 0;
}

std::vector<Cand> candidates(const Scene& s, const std::vector<Edge>& E, const Cam& c, int mode) {
  std::vector<Cand> out;
  for (size_t i = 0; i < E.size(); ++i) {
    const Edge& e = E[i];
    bool take = true;
    if (mode == 0 && e.nf == 2) take = facing(s, e.f[0], c.eye) != facing(s, e.f[1], c.eye);
    if (!take) continue;
    double ax, ay, bx, by;
    if (!project(c, s.vert[e.a], ax, ay) || !project(c, s.vert[e.b], bx, by)) continue;
    double dx = bx - ax, dy = by - ay;
    double t0 = 0, t1 = 1;
    double pp[4] = {-dx, dx, -dy, dy};
    double qq[4] = {ax, c.W - ax, ay, c.H - ay};
    bool ok = true;
    for (int k = 0; k < 4 && ok; ++k) {
      if (pp[k] == 0) { if (qq[k] < 0) ok = false; continue; }
      double r = qq[k] / pp[k];
      if (pp[k] < 0) t0 = std::max(t0, r); else t1 = std::min(t1, r);
    }
    if (!ok || !(t1 > t0)) continue;
    double L = std::sqrt(dx * dx + dy * dy) * (t1 - t0);
    if (!(L > 0)) continue;
    out.push_back(Cand{(int)i, t0, t1, L, {ax, ay, 0}, {bx, by, 0}});
  }
  return out;
}

}  // namespace

// ==================================================================== C API
extern "C" {

void orc_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out) {
  U4 c = {{ctr[0], ctr[1], ctr[2], ctr[3]}};
  U4 r = philox4x32_10(c, key[0], key[1]);
  for (int i = 0; i < 4; ++i) out[i] = r.w[i];
}

int orc_env_alias(const float* rgb, int w, int h, double* prob, int* alias, double* pmf) {
  std::vector<double> p, q; std::vector<int> a;
  if (build_alias(rgb, w, h, p, a, q)) return 1;
  std::copy(p.begin(), p.end(), prob);
  std::copy(a.begin(), a.end(), alias);
  std::copy(q.begin(), q.end(), pmf);
  return 0;
}

int orc_alias_pick(const double* prob, const int* alias, int n, uint32_t u0, uint32_t u1) {
  return alias_pick(prob, alias, n, u0, u1);
}

long long orc_mesh_color_index(int r, long long t, double alpha, double beta) {
  // Sec. 3.3: k = (t (r+1)(r+2) + i (2r - i + 3)) / 2 + j, (i, j) = floor(r (alpha, beta)).
  long long i = (long long)std::floor(r * alpha), j = (long long)std::floor(r * beta);
  return (t * (r + 1) * (r + 2) + i * (2LL * r - i + 3)) / 2 + j;
}

static Mat mat_from(const double* p5) {
  Mat m;
  for (int c = 0; c < 3; ++c) m.kd[c] = p5[c];
  for (int c = 0; c < 3; ++c) m.ks[c] = p5[3];
  m.alpha = p5[4];
  return m;
}

void orc_brdf_eval(int brdf, int fresnel, const double* p5, const double* n, const double* wi, const double* wo,
                   double* out) {
  Mat m = mat_from(p5);
  MatT<double> mt;
  for (int c = 0; c < 3; ++c) { mt.kd[c] = m.kd[c]; mt.ks[c] = m.ks[c]; }
  mt.alpha = m.alpha;
  V3d N{n[0], n[1], n[2]}, I{wi[0], wi[1], wi[2]}, O{wo[0], wo[1], wo[2]};
  brdf_eval(brdf, fresnel, mt, N, I, O, out);
}

double orc_brdf_pdf(int brdf, const double* p5, const double* n, const double* wi, const double* wo) {
  V3d N{n[0], n[1], n[2]}, I{wi[0], wi[1], wi[2]}, O{wo[0], wo[1], wo[2]};
  return brdf_pdf(brdf, mat_from(p5), N, I, O);
}

double orc_brdf_sample(int brdf, const double* p5, const double* n, const double* wo, double ul, double u1,
                       double u2, double* wi) {
  V3d N{n[0], n[1], n[2]}, O{wo[0], wo[1], wo[2]}, I{0, 0, 0};
  double pdf = brdf_sample(brdf, mat_from(p5), N, O, ul, u1, u2, I, nullptr);
  wi[0] = I.x; wi[1] = I.y; wi[2] = I.z;
  return pdf;
}

void orc_closest_hit(const orc_scene* in, const double* rays, int n, int exclude, int* out_tri, double* out_t) {
  Scene s;
  if (!load_scene(in, s)) return;
  parallel_for(n, (int)std::thread::hardware_concurrency(), [&](int, int i) {
    const double* r = rays + 7 * (size_t)i;
    Hit h = closest(s, V3d{r[0], r[1], r[2]}, V3d{r[3], r[4], r[5]}, exclude, r[6]);
    out_tri[i] = h.tri;
    out_t[i] = h.tri >= 0 ? h.t : INFINITY;
  });
}

static bool check_common(const orc_view* views, int n_views, const orc_params* p) {
  if (!views || n_views <= 0 || !p || p->max_bounces < 1 || p->max_bounces > MAX_B) return false;
  if (p->secondary < 0 || p->secondary > 2) return false;
  for (int v = 0; v < n_views; ++v)
    if (views[v].width <= 0 || views[v].height <= 0 || views[v].spp <= 0 || views[v].n_lights < 0 ||
        views[v].n_lights > 2)
      return false;
  return true;
}

static Rng rng_of(const orc_params* p) {
  return Rng{(uint32_t)(p->seed & 0xffffffffu), (uint32_t)(p->seed >> 32)};
}

long long orc_render_pixels(const orc_scene* in, const orc_view* views, int n_views, const orc_params* p,
                            const int* pix, int n, double* out) {
  Scene s;
  if (!load_scene(in, s) || !check_common(views, n_views, p)) return -1;
  Rng rng = rng_of(p);
  int nt = nthreads(p);
  std::vector<long long> seg(nt, 0);
  for (int i = 0; i < n; ++i)
    if (pix[3 * i] < 0 || pix[3 * i] >= n_views) return -1;
  parallel_for(n, nt, [&](int tid, int i) {
    const orc_view& v = views[pix[3 * i]];
    Cam c = make_cam(v, s);
    int x = pix[3 * i + 1], y = pix[3 * i + 2];
    uint32_t c0 = c.off + (uint32_t)(y * c.W + x);
    double acc[3] = {0, 0, 0};
    for (int sidx = 0; sidx < c.spp; ++sidx) {
      U4 u = rng.draw(c0, (uint32_t)sidx, 0u, 0u);
      V3d d = cam_dir(c, x + unif(u.w[0]), y + unif(u.w[1]));
      double L[3];
      trace_path<double>(s, rng, p->max_bounces, c.lt, c.eye, d, c0, (uint32_t)sidx, 0u, nullptr, L, seg[tid]);
      for (int k = 0; k < 3; ++k) acc[k] += L[k];
    }
    for (int k = 0; k < 3; ++k) out[3 * i + k] = acc[k] / c.spp;
  });
  long long tot = 0;
  for (auto x : seg) tot += x;
  return tot;
}

long long orc_render_signatures(const orc_scene* in, const orc_view* views, int n_views, const orc_params* p,
                                const int* pix, int n, uint64_t* out) {
  Scene s;
  if (!load_scene(in, s) || !check_common(views, n_views, p)) return -1;
  for (int i = 0; i < n; ++i)
    if (pix[3 * i] < 0 || pix[3 * i] >= n_views) return -1;
  Rng rng = rng_of(p);
  int nt = nthreads(p);
  std::vector<long long> seg(nt, 0);
  parallel_for(n, nt, [&](int tid, int i) {
    const orc_view& v = views[pix[3 * i]];
    Cam c = make_cam(v, s);
    int x = pix[3 * i + 1], y = pix[3 * i + 2];
    uint32_t c0 = c.off + (uint32_t)(y * c.W + x);
    uint64_t acc = 0;
    for (int sidx = 0; sidx < c.spp; ++sidx) {
      U4 u = rng.draw(c0, (uint32_t)sidx, 0u, 0u);
      V3d d = cam_dir(c, x + unif(u.w[0]), y + unif(u.w[1]));
      double L[3];
      uint64_t h = 0;
      trace_path<double>(s, rng, p->max_bounces, c.lt, c.eye, d, c0, (uint32_t)sidx, 0u, nullptr, L, seg[tid],
                         nullptr, nullptr, 0, -1, &h);
      acc += h;
    }
    out[i] = acc;
  });
  long long tot = 0;
  for (auto x : seg) tot += x;
  return tot;
}

long long orc_grad_pixels(const orc_scene* in, const orc_view* views, int n_views, const orc_params* p,
                          const int* pix, int n, const double* dLdI, double* d_verts, double* d_face) {
  g_dual_overflow = false;
  Scene s;
  if (!load_scene(in, s) || !check_common(views, n_views, p)) return -1;
  Rng rng = rng_of(p);
  int nt = nthreads(p);
  std::vector<long long> seg(nt, 0);
  std::vector<std::vector<double>> gv(nt, std::vector<double>(3 * (size_t)s.nv, 0.0));
  std::vector<std::vector<double>> gf(nt, std::vector<double>((size_t)s.np * s.nf * s.ntex, 0.0));
  std::vector<Edge> E;
  EdgeTree T;
  if (p->secondary) E = edge_list(s);
  if (p->secondary == 2) T = edge_tree(s, E);
  SecCtx sc{&E, p->edge_mode, p->secondary, &T};
  const SecCtx* sec = p->secondary ? &sc : nullptr;
  parallel_for(n, nt, [&](int tid, int i) {
    const double* w = dLdI + 3 * (size_t)i;
    if (w[0] == 0 && w[1] == 0 && w[2] == 0) return;
    const orc_view& v = views[pix[3 * i]];
    Cam c = make_cam(v, s);
    int x = pix[3 * i + 1], y = pix[3 * i + 2];
    uint32_t c0 = c.off + (uint32_t)(y * c.W + x);
    for (int sidx = 0; sidx < c.spp; ++sidx) {
      U4 u = rng.draw(c0, (uint32_t)sidx, 0u, 0u);
      V3d d = cam_dir(c, x + unif(u.w[0]), y + unif(u.w[1]));
      Vars vars;
      Dual L[3];
      trace_path<Dual>(s, rng, p->max_bounces, c.lt, c.eye, d, c0, (uint32_t)sidx, 0u, &vars, L, seg[tid], nullptr, sec);
      Dual loss = L[0] * (w[0] / c.spp) + L[1] * (w[1] / c.spp) + L[2] * (w[2] / c.spp);
      scatter_grad(s, vars, loss, gv[tid].data(), gf[tid].data(), s.np);
    }
  });
  for (int t = 0; t < nt; ++t) {
    for (size_t k = 0; k < gv[t].size(); ++k) d_verts[k] += gv[t][k];
    if (d_face) for (size_t k = 0; k < gf[t].size(); ++k) d_face[k] += gf[t][k];
  }
  if (g_dual_overflow) return -1;
  long long tot = 0;
  for (auto x : seg) tot += x;
  return tot;
}

int orc_edge_candidates(const orc_scene* in, const orc_view* view, const orc_params* p, int* out_edges) {
  Scene s;
  if (!load_scene(in, s) || !view || !p) return -1;
  std::vector<Edge> E = edge_list(s);
  std::vector<Cand> C = candidates(s, E, make_cam(*view, s), p->edge_mode);
  if (out_edges)
    for (size_t i = 0; i < C.size(); ++i) { out_edges[2 * i] = E[C[i].e].a; out_edges[2 * i + 1] = E[C[i].e].b; }
  return (int)C.size();
}

long long orc_edge_grad(const orc_scene* in, const orc_view* views, int n_views, const orc_params* p,
                        const double* dLdI, double* d_verts) {
  Scene s;
  if (!load_scene(in, s) || !check_common(views, n_views, p)) return -1;
  Rng rng = rng_of(p);
  int nt = nthreads(p);
  std::vector<Edge> E = edge_list(s);
  std::vector<long long> seg(nt, 0);
  std::vector<std::vector<double>> gv(nt, std::vector<double>(3 * (size_t)s.nv, 0.0));
  for (int vi = 0; vi < n_views; ++vi) {
    Cam c = make_cam(views[vi], s);
    std::vector<Cand> C = candidates(s, E, c, p->edge_mode);
    if (C.empty()) continue;
    long long spp_e = p->edge_spp > 0 ? p->edge_spp : c.spp;
    long long Ne = (long long)c.W * c.H * spp_e;
    uint64_t ncand = C.size();
    // samples are split across threads in contiguous blocks
    int nblk = nt * 8;
    parallel_for(nblk, nt, [&](int tid, int blk) {
      long long k0 = Ne * blk / nblk, k1 = Ne * (blk + 1) / nblk;
      for (long long k = k0; k < k1; ++k) {
        U4 u = rng.draw((uint32_t)k, c.off, 0u, 1u);
        // stratified: sample k draws uniformly from the integers [k*n, (k+1)*n) and
        // integer t selects candidate t / N_e, so each candidate has probability 1/n
        uint64_t t = (uint64_t)k * ncand + (((uint64_t)(u.w[0] >> 8) * ncand) >> 24);
        const Cand& cd = C[(size_t)(t / (uint64_t)Ne)];
        double tau = cd.t0 + unif(u.w[1]) * (cd.t1 - cd.t0);
        double sx = cd.sa.x + (cd.sb.x - cd.sa.x) * tau, sy = cd.sa.y + (cd.sb.y - cd.sa.y) * tau;
        int x = (int)std::floor(sx), y = (int)std::floor(sy);
        if (x < 0 || y < 0 || x >= c.W || y >= c.H) continue;
        const double* w = dLdI + 3 * ((size_t)c.off + (size_t)y * c.W + x);
        if (w[0] == 0 && w[1] == 0 && w[2] == 0) continue;
        double ex = cd.sb.x - cd.sa.x, ey = cd.sb.y - cd.sa.y;
        double el = std::sqrt(ex * ex + ey * ey);
        double nx = -ey / el, ny = ex / el;
        double Lm[3], Lp[3];
        trace_path<double>(s, rng, p->max_bounces, c.lt, c.eye, cam_dir(c, sx - EDGE_EPS * nx, sy - EDGE_EPS * ny),
                           (uint32_t)k, c.off, 2u, nullptr, Lm, seg[tid]);
        trace_path<double>(s, rng, p->max_bounces, c.lt, c.eye, cam_dir(c, sx + EDGE_EPS * nx, sy + EDGE_EPS * ny),
                           (uint32_t)k, c.off, 2u, nullptr, Lp, seg[tid]);
        double g = 0;
        for (int ch = 0; ch < 3; ++ch) g += w[ch] * (Lm[ch] - Lp[ch]);
        if (g == 0) continue;
        double wt = g * (double)ncand * cd.len / (double)Ne;
        const Edge& e = E[cd.e];
        V3d ja = proj_jt(c, s.vert[e.a], nx, ny), jb = proj_jt(c, s.vert[e.b], nx, ny);
        double* G = gv[tid].data();
        G[3 * e.a] += wt * (1 - tau) * ja.x; G[3 * e.a + 1] += wt * (1 - tau) * ja.y; G[3 * e.a + 2] += wt * (1 - tau) * ja.z;
        G[3 * e.b] += wt * tau * jb.x; G[3 * e.b + 1] += wt * tau * jb.y; G[3 * e.b + 2] += wt * tau * jb.z;
      }
    });
  }
  for (int t = 0; t < nt; ++t)
    for (size_t k = 0; k < gv[t].size(); ++k) d_verts[k] += gv[t][k];
  long long tot = 0;
  for (auto x : seg) tot += x;
  return tot;
}

// Shadow-edge term (point lights, shadows on surfaces the camera sees). A
// point light's shadow on a visible surface ends where light rays graze the
// edges that are silhouettes seen from the light; in the image that boundary is
// the projection, through the receiving surface, of those edges, and moving the
// occluder or the receiver moves it. Per view and per light l: candidates =
// edges whose two faces face the light on opposite sides (or boundary edges),
// in edge order; N = W*H*spp samples (edge_spp overrides spp); sample k picks
// candidate t/N for t uniform in [k n, (k+1) n) and tau uniform on the edge
// (counter (k, pixel_offset, l<<4, 3)); y = A + tau (B - A); the light ray from
// L through y, continued from y + SH_EDGE_DELTA |y - L| along it, finds the
// receiver point q = L + s (y - L) on a face other than the edge's own (that
// ray meets their planes only at y, so they receive no shadow from the edge);
// S = q projected to the view. Camera paths
// at S -+ EDGE_EPS n_S (counters (k, pixel_offset, b<<4|call, 4 + l)), n_S the
// screen normal of the boundary curve S(tau), give L- - L+. The boundary moves
// with the occluder (dq = s P dy, P = I - u n_r^T / n_r.u, u = y - L) and with
// the receiver plane; its screen-normal speed is n_S . J_proj(q) dq. The
// sample adds <dL/dI_S, L- - L+> n_cand |dS/dtau| / N times that speed.
long long orc_shadow_edge_grad(const orc_scene* in, const orc_view* views, int n_views, const orc_params* p,
                               const double* dLdI, double* d_verts) {
  g_dual_overflow = false;
  Scene s;
  if (!load_scene(in, s) || !check_common(views, n_views, p)) return -1;
  Rng rng = rng_of(p);
  int nt = nthreads(p);
  std::vector<Edge> E = edge_list(s);
  std::vector<long long> seg(nt, 0);
  std::vector<std::vector<double>> gv(nt, std::vector<double>(3 * (size_t)s.nv, 0.0));
  for (int vi = 0; vi < n_views; ++vi) {
    Cam c = make_cam(views[vi], s);
    long long spp_e = p->edge_spp > 0 ? p->edge_spp : c.spp;
    long long N = (long long)c.W * c.H * spp_e;
    for (size_t l = 0; l < c.lt.pos.size(); ++l) {
      V3d L = c.lt.pos[l];
      std::vector<int> cand;
      for (size_t i = 0; i < E.size(); ++i) {
        const Edge& e = E[i];
        if (e.nf == 2 && facing(s, e.f[0], L) == facing(s, e.f[1], L)) continue;
        cand.push_back((int)i);
      }
      if (cand.empty()) continue;
      uint64_t ncand = cand.size();
      int nblk = nt * 8;
      parallel_for(nblk, nt, [&](int tid, int blk) {
        long long k0 = N * blk / nblk, k1 = N * (blk + 1) / nblk;
        for (long long k = k0; k < k1; ++k) {
          U4 u = rng.draw((uint32_t)k, c.off, (uint32_t)l << 4, 3u);
          uint64_t t = (uint64_t)k * ncand + (((uint64_t)(u.w[0] >> 8) * ncand) >> 24);
          const Edge& e = E[cand[(size_t)(t / (uint64_t)N)]];
          double tau = unif(u.w[1]);
          V3d A = s.vert[e.a], Bv = s.vert[e.b];
          V3d y = A + scl(Bv - A, tau);
          V3d uvec = y - L;
          double dy = len(uvec);
          if (!(dy > 0)) continue;
          V3d dir = scl(uvec, 1.0 / dy);
          V3d org = y + scl(dir, SH_EDGE_DELTA * dy);
          ++seg[tid];
          Hit h = closest(s, org, dir, e.f[0], INFINITY, e.nf == 2 ? e.f[1] : -1);
          if (h.tri < 0) continue;
          V3d q = org + scl(dir, h.t);
          double sx, sy;
          if (!project(c, q, sx, sy)) continue;
          int x = (int)std::floor(sx), yy = (int)std::floor(sy);
          if (x < 0 || yy < 0 || x >= c.W || yy >= c.H) continue;
          const double* w = dLdI + 3 * ((size_t)c.off + (size_t)yy * c.W + x);
          if (w[0] == 0 && w[1] == 0 && w[2] == 0) continue;
          // screen tangent of the boundary curve: dS/dtau = J_proj(q) s P (B - A)
          const int* rf = &s.face[3 * h.tri];
          V3d nr = cross(s.vert[rf[1]] - s.vert[rf[0]], s.vert[rf[2]] - s.vert[rf[0]]);
          double nu = dot(nr, uvec);
          if (!(std::fabs(nu) > 0)) continue;
          double sc = len(q - L) / dy;
          V3d ab = Bv - A;
          V3d dq = scl(ab - scl(uvec, dot(nr, ab) / nu), sc);
          V3d jx = proj_jt(c, q, 1.0, 0.0), jy = proj_jt(c, q, 0.0, 1.0);
          double tx = dot(jx, dq), ty = dot(jy, dq);
          double lt = std::sqrt(tx * tx + ty * ty);
          if (!(lt > 0)) continue;
          double nx = -ty / lt, ny = tx / lt;
          double Lm[3], Lp[3];
          trace_path<double>(s, rng, p->max_bounces, c.lt, c.eye, cam_dir(c, sx - EDGE_EPS * nx, sy - EDGE_EPS * ny),
                             (uint32_t)k, c.off, 4u + (uint32_t)l, nullptr, Lm, seg[tid]);
          trace_path<double>(s, rng, p->max_bounces, c.lt, c.eye, cam_dir(c, sx + EDGE_EPS * nx, sy + EDGE_EPS * ny),
                             (uint32_t)k, c.off, 4u + (uint32_t)l, nullptr, Lp, seg[tid]);
          double g = 0;
          for (int ch = 0; ch < 3; ++ch) g += w[ch] * (Lm[ch] - Lp[ch]);
          if (g == 0) continue;
          double wt = g * (double)ncand * lt / (double)N;
          // the boundary's screen-normal speed, through dual numbers of the occluder's
          // edge and the receiver's vertices: q = L + s (y - L) on the receiver plane
          Vars vars;
          using DA = Access<Dual>;
          V3<Dual> Ad = DA::vertex(s, &vars, e.a), Bd = DA::vertex(s, &vars, e.b);
          V3<Dual> r0 = DA::vertex(s, &vars, rf[0]), r1 = DA::vertex(s, &vars, rf[1]), r2 = DA::vertex(s, &vars, rf[2]);
          V3<Dual> yd = scl(Ad, 1.0 - tau) + scl(Bd, tau);
          V3<Dual> Ld = lift<Dual>(L);
          V3<Dual> ud = yd - Ld;
          V3<Dual> nd = cross(r1 - r0, r2 - r0);
          Dual sd = dot(nd, r0 - Ld) / dot(nd, ud);
          V3<Dual> qd = Ld + scl(ud, sd);
          V3d js = scl(jx, nx) + scl(jy, ny);
          Dual vn = dot(lift<Dual>(js), qd - lift<Dual>(q));
          scatter_grad(s, vars, vn * wt, gv[tid].data(), nullptr, s.np);
        }
      });
    }
  }
  for (int t = 0; t < nt; ++t)
    for (size_t k = 0; k < gv[t].size(); ++k) d_verts[k] += gv[t][k];
  if (g_dual_overflow) return -1;
  long long tot = 0;
  for (auto x : seg) tot += x;
  return tot;
}

long long orc_trace_screen(const orc_scene* in, const orc_view* view, const orc_params* p, double px, double py,
                           uint32_t c0, uint32_t c1, uint32_t stream, double* rgb, const double* grad_w,
                           double* d_verts, double* d_face) {
  g_dual_overflow = false;
  Scene s;
  if (!load_scene(in, s) || !check_common(view, 1, p)) return -1;
  Rng rng = rng_of(p);
  Cam c = make_cam(*view, s);
  V3d d = cam_dir(c, px, py);
  long long seg = 0;
  if (!grad_w) {
    trace_path<double>(s, rng, p->max_bounces, c.lt, c.eye, d, c0, c1, stream, nullptr, rgb, seg);
    return seg;
  }
  Vars vars;
  Dual L[3];
  std::vector<Edge> E;
  EdgeTree T;
  if (p->secondary) E = edge_list(s);
  if (p->secondary == 2) T = edge_tree(s, E);
  SecCtx sc{&E, p->edge_mode, p->secondary, &T};
  trace_path<Dual>(s, rng, p->max_bounces, c.lt, c.eye, d, c0, c1, stream, &vars, L, seg, nullptr,
                   p->secondary ? &sc : nullptr);
  for (int k = 0; k < 3; ++k) rgb[k] = L[k].v;
  Dual loss = L[0] * grad_w[0] + L[1] * grad_w[1] + L[2] * grad_w[2];
  scatter_grad(s, vars, loss, d_verts, d_face, s.np);
  if (g_dual_overflow) return -1;
  return seg;
}

int orc_sec_edge_pmf(const orc_scene* in, const double* p, const double* n, double bnd, int edge_mode, double* pmf) {
  Scene s;
  if (!load_scene(in, s)) return -1;
  std::vector<Edge> E = edge_list(s);
  EdgeTree t = edge_tree(s, E);
  V3d pv{p[0], p[1], p[2]}, nv{n[0], n[1], n[2]};
  for (int leaf = 0; leaf < t.nleaf; ++leaf) {
    size_t k = ((size_t)1 << t.L) + leaf;
    double pr = 1.0;
    for (size_t c = k; c > 1; c /= 2) {
      size_t par = c / 2;
      double wa = tree_weight(t, 2 * par, pv, nv, bnd, edge_mode == 0),
             wb = tree_weight(t, 2 * par + 1, pv, nv, bnd, edge_mode == 0);
      pr *= wa + wb > 0 ? (c % 2 == 0 ? wa : wb) / (wa + wb) : 0.0;
    }
    int first = leaf * t.G, cnt = std::min(t.G, t.nE - first);
    for (int e = first; e < first + cnt; ++e) pmf[e] = pr / cnt;
  }
  return (int)E.size();
}

int orc_sec_edge_picks(const orc_scene* in, unsigned long long seed, uint32_t c1, int b, uint32_t stream,
                       const double* p, const double* n, double bnd, int edge_mode, const uint32_t* uleaf, int count,
                       int* edge, double* prob) {
  Scene s;
  if (!load_scene(in, s) || count < 0) return -1;
  std::vector<Edge> E = edge_list(s);
  EdgeTree t = edge_tree(s, E);
  Rng rng{(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
  V3d pv{p[0], p[1], p[2]}, nv{n[0], n[1], n[2]};
  for (int i = 0; i < count; ++i)
    edge[i] = tree_pick(t, rng, (uint32_t)i, c1, b, stream, pv, nv, bnd, edge_mode == 0, uleaf[i], prob[i]);
  return count;
}

long long orc_trace_screen_taped(const orc_scene* in, const orc_view* view, const orc_params* p, double px,
                                 double py, uint32_t c0, uint32_t c1, uint32_t stream, int mode, double* tape,
                                 int* tape_len, double* rgb) {
  Scene s;
  if (!load_scene(in, s) || !check_common(view, 1, p) || !tape_len) return -1;
  Rng rng = rng_of(p);
  Cam c = make_cam(*view, s);
  Tape tp;
  tp.mode = mode;
  if (mode == 2) tp.v.assign(tape, tape + *tape_len);
  long long seg = 0;
  trace_path<double>(s, rng, p->max_bounces, c.lt, c.eye, cam_dir(c, px, py), c0, c1, stream, nullptr, rgb, seg, &tp);
  if (tp.bad || (mode == 2 && tp.pos != tp.v.size())) return -2;
  if (mode == 1) {
    if ((int)tp.v.size() > *tape_len) return -3;
    std::copy(tp.v.begin(), tp.v.end(), tape);
    *tape_len = (int)tp.v.size();
  }
  return seg;
}

void orc_microfacet(int brdf, double alpha, double c, double* D, double* G1) {
  *D = D_fn(brdf, c, clamp_alpha(alpha));
  *G1 = G1_fn(brdf, c, clamp_alpha(alpha));
}

}  // extern "C"

// Device-side building blocks of the path tracer: vector math, Philox4x32-10,
// pinhole camera, watertight ray/triangle test, environment lookup and alias
// sampling, and the Torrance-Sparrow BRDF (value, pdf, sampling, adjoint).
//
// The material is the paper's Torrance-Sparrow model with diffuse albedo,
// specular and roughness per mesh facet (Sec. 3.3 "Representation"; mesh
// colors at r = 0, so the texel of face t is t). The exact conventions (Fresnel
// factor held at its normal-incidence value ks, alpha = roughness clamped to
// [0.01, 1], separable Smith G1, one-sample lobe mixture) are the readings the
// whole library follows.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace st {

constexpr float PI_F = 3.14159265358979323846f;
constexpr float T_EPS = 1e-5f;      // closest/any hit accepts t > T_EPS
constexpr float Z_NEAR = 1e-4f;     // edge endpoints closer than this to the eye plane are skipped
constexpr float EDGE_EPS = 1e-3f;   // side offset of edge samples, in pixels
constexpr int MAX_LIGHTS = 8;
constexpr int MAX_B = 8;

// ------------------------------------------------------------------ vectors
__host__ __device__ __forceinline__ float3 mk3(float x, float y, float z) { return make_float3(x, y, z); }
__host__ __device__ __forceinline__ float3 operator+(float3 a, float3 b) { return mk3(a.x + b.x, a.y + b.y, a.z + b.z); }
__host__ __device__ __forceinline__ float3 operator-(float3 a, float3 b) { return mk3(a.x - b.x, a.y - b.y, a.z - b.z); }
__host__ __device__ __forceinline__ float3 operator-(float3 a) { return mk3(-a.x, -a.y, -a.z); }
__host__ __device__ __forceinline__ float3 operator*(float3 a, float s) { return mk3(a.x * s, a.y * s, a.z * s); }
__host__ __device__ __forceinline__ float3 operator*(float s, float3 a) { return mk3(a.x * s, a.y * s, a.z * s); }
__host__ __device__ __forceinline__ float3 mul(float3 a, float3 b) { return mk3(a.x * b.x, a.y * b.y, a.z * b.z); }
__host__ __device__ __forceinline__ float3& operator+=(float3& a, float3 b) { a.x += b.x; a.y += b.y; a.z += b.z; return a; }
__host__ __device__ __forceinline__ float3& operator-=(float3& a, float3 b) { a.x -= b.x; a.y -= b.y; a.z -= b.z; return a; }
__host__ __device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__host__ __device__ __forceinline__ float3 cross3(float3 a, float3 b) {
  return mk3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float len3(float3 a) { return sqrtf(dot3(a, a)); }
__device__ __forceinline__ float3 norm3(float3 a) { float l = len3(a); return mk3(a.x / l, a.y / l, a.z / l); }
__device__ __forceinline__ float3 xyz(float4 a) { return mk3(a.x, a.y, a.z); }
__device__ __forceinline__ float comp3(float3 a, int k) { return k == 0 ? a.x : (k == 1 ? a.y : a.z); }

// ------------------------------------------------------------------ Philox4x32-10
// Counter-based generator of Salmon et al. (SC'11): ten rounds of two 32x32
// multiplies whose high halves are xored into the other words with the round
// key; the key advances by the golden-ratio and sqrt(3)-1 Weyl increments.
struct U4 { uint32_t x, y, z, w; };

__device__ __forceinline__ U4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
  }
  return U4{c0, c1, c2, c3};
}
// 24-bit uniform in [0, 1): exact in single precision.
__device__ __forceinline__ float unif(uint32_t x) { return (float)(x >> 8) * (1.0f / 16777216.0f); }

struct Key { uint32_t k0, k1; };

// ------------------------------------------------------------------ camera
struct DevView {
  float3 eye, fwd, right, up;
  float kx, ky;            // tan(fov/2) * aspect, tan(fov/2)
  int W, H, spp;
  uint32_t off;            // low 32 bits of pixel_offset (counter word)
  long long pix_off;       // packed-image row of pixel (0, 0)
  long long bin_base;      // first pixel of the view in the call's pixel space (accumulation)
  long long bin_cell;      // first cell of the view in the primary-visibility bins
  int kb;                  // bin cells per pixel side (1, 2, 4 or 8)
  int nvl;                 // the view's own point lights (after the scene's)
  float4 vl[4];            // (position, 0), (intensity, 0) per view light
};

__device__ __forceinline__ float3 cam_dir(const DevView& v, float px, float py) {
  float sx = 2.0f * px / (float)v.W - 1.0f;
  float sy = 1.0f - 2.0f * py / (float)v.H;
  return norm3(v.fwd + v.right * (sx * v.kx) + v.up * (sy * v.ky));
}

// pixel coordinates of X; false if X is not in front of the eye
__device__ __forceinline__ bool cam_project(const DevView& v, float3 X, float& px, float& py) {
  float3 rel = X - v.eye;
  float z = dot3(rel, v.fwd);
  if (!(z > Z_NEAR)) return false;
  float sx = dot3(rel, v.right) / (z * v.kx);
  float sy = dot3(rel, v.up) / (z * v.ky);
  px = (sx + 1.0f) * (float)v.W * 0.5f;
  py = (1.0f - sy) * (float)v.H * 0.5f;
  return true;
}

// d(px, py)/dX contracted with the screen direction (nx, ny)
__device__ __forceinline__ float3 cam_project_jt(const DevView& v, float3 X, float nx, float ny) {
  float3 rel = X - v.eye;
  float z = dot3(rel, v.fwd);
  float sx = dot3(rel, v.right) / (z * v.kx);
  float sy = dot3(rel, v.up) / (z * v.ky);
  float3 dpx = (v.right - v.fwd * (sx * v.kx)) * ((float)v.W * 0.5f / (z * v.kx));
  float3 dpy = (v.up - v.fwd * (sy * v.ky)) * (-(float)v.H * 0.5f / (z * v.ky));
  return dpx * nx + dpy * ny;
}

// ------------------------------------------------------------------ watertight ray/triangle
// Woop, Benthin and Wald, "Watertight Ray/Triangle Intersection" (JCGT 2013):
// shear so the ray is +z, test the signs of the three 2-D edge functions, and
// redo them in double when one is exactly zero.
struct RayPre {
  float3 o;
  int kx, ky, kz;
  float sx, sy, sz;
};

__device__ __forceinline__ RayPre ray_pre(float3 o, float3 d) {
  RayPre r;
  r.o = o;
  float ax = fabsf(d.x), ay = fabsf(d.y), az = fabsf(d.z);
  int kz = (ax > ay) ? (ax > az ? 0 : 2) : (ay > az ? 1 : 2);
  int kx = kz == 2 ? 0 : kz + 1;
  int ky = kx == 2 ? 0 : kx + 1;
  float dz = comp3(d, kz);
  if (dz < 0.0f) { int t = kx; kx = ky; ky = t; }
  r.kx = kx; r.ky = ky; r.kz = kz;
  r.sz = 1.0f / dz;
  r.sx = comp3(d, kx) * r.sz;
  r.sy = comp3(d, ky) * r.sz;
  return r;
}

// returns t (> T_EPS and < tmax) or a negative value on a miss
__device__ __forceinline__ float tri_test(const RayPre& r, float3 p0, float3 p1, float3 p2, float tmax) {
  float3 A = p0 - r.o, B = p1 - r.o, C = p2 - r.o;
  float Akz = comp3(A, r.kz), Bkz = comp3(B, r.kz), Ckz = comp3(C, r.kz);
  float Ax = comp3(A, r.kx) - r.sx * Akz, Ay = comp3(A, r.ky) - r.sy * Akz;
  float Bx = comp3(B, r.kx) - r.sx * Bkz, By = comp3(B, r.ky) - r.sy * Bkz;
  float Cx = comp3(C, r.kx) - r.sx * Ckz, Cy = comp3(C, r.ky) - r.sy * Ckz;
  float U = Cx * By - Cy * Bx, V = Ax * Cy - Ay * Cx, W = Bx * Ay - By * Ax;
  if (U == 0.0f || V == 0.0f || W == 0.0f) {
    U = (float)((double)Cx * (double)By - (double)Cy * (double)Bx);
    V = (float)((double)Ax * (double)Cy - (double)Ay * (double)Cx);
    W = (float)((double)Bx * (double)Ay - (double)By * (double)Ax);
  }
  if ((U < 0.0f || V < 0.0f || W < 0.0f) && (U > 0.0f || V > 0.0f || W > 0.0f)) return -1.0f;
  float det = U + V + W;
  if (det == 0.0f) return -1.0f;
  float T = U * (r.sz * Akz) + V * (r.sz * Bkz) + W * (r.sz * Ckz);
  float t = T / det;
  return (t > T_EPS && t < tmax) ? t : -1.0f;
}

// ------------------------------------------------------------------ environment
struct DevEnv {
  int w, h;                 // 0 = no environment
  const float4* tex;        // [h*w] (r, g, b, pmf)
  const float2* alias;      // [h*w] (prob, alias index as int bits)
  float pdf_scale;          // N / (2 pi^2)
};

__device__ __forceinline__ int env_texel(const DevEnv& e, float3 d, float& sin_t) {
  float phi = atan2f(d.x, -d.z) + PI_F;
  int col = (int)(phi * (1.0f / (2.0f * PI_F)) * (float)e.w);
  col = min(max(col, 0), e.w - 1);
  float th = acosf(fminf(fmaxf(d.y, -1.0f), 1.0f));
  int row = (int)(th * (1.0f / PI_F) * (float)e.h);
  row = min(max(row, 0), e.h - 1);
  sin_t = sqrtf(fmaxf(0.0f, 1.0f - d.y * d.y));
  return row * e.w + col;
}

__device__ __forceinline__ float env_pdf(const DevEnv& e, float pmf, float sin_t) {
  return sin_t > 0.0f ? pmf * e.pdf_scale / sin_t : 0.0f;
}

// alias-table texel choice from two raw words (integer bin, 24-bit coin)
__device__ __forceinline__ int env_pick(const DevEnv& e, uint32_t u0, uint32_t u1) {
  uint32_t N = (uint32_t)(e.w * e.h);
  int bin = (int)(((uint64_t)(u0 >> 8) * (uint64_t)N) >> 24);
  float2 a = __ldg(&e.alias[bin]);
  return unif(u1) < a.x ? bin : __float_as_int(a.y);
}

// ------------------------------------------------------------------ BRDF
// kd and ks per channel (a scalar specular is stored in all three), roughness
struct Mat { float kd[3]; float ks[3]; float alpha; };

// specular lobe probability: mean ks over mean ks + mean kd, clamped
__device__ __forceinline__ float lobe_prob(const Mat& m) {
  float ks = (m.ks[0] + m.ks[1] + m.ks[2]) * (1.0f / 3.0f);
  float den = ks + (m.kd[0] + m.kd[1] + m.kd[2]) * (1.0f / 3.0f);
  if (!(den > 0.0f)) return 0.5f;
  return fminf(fmaxf(ks / den, 0.05f), 0.95f);
}

__device__ __forceinline__ float clamp_alpha(float a, bool& clamped) {
  clamped = !(a >= 0.01f && a <= 1.0f);
  return fminf(fmaxf(a, 0.01f), 1.0f);
}

// D and its partials in c = cos(theta_h) and alpha
__device__ __forceinline__ float D_eval(int brdf, float c, float a, float* dc = nullptr, float* da = nullptr) {
  if (brdf == 0) {  // GGX
    float a2 = a * a;
    float k = c * c * (a2 - 1.0f) + 1.0f;
    float D = a2 / (PI_F * k * k);
    if (dc) *dc = -4.0f * a2 * c * (a2 - 1.0f) / (PI_F * k * k * k);
    if (da) *da = 2.0f * a / (PI_F * k * k) * (1.0f - 2.0f * a2 * c * c / k);
    return D;
  }
  float c2 = c * c;
  float a2 = a * a;
  float tan2 = (1.0f - c2) / c2;
  float D = expf(-tan2 / a2) / (PI_F * a2 * c2 * c2);
  if (dc) *dc = D * (2.0f / (a2 * c2 * c) - 4.0f / c);
  if (da) *da = D * (2.0f * tan2 / (a2 * a) - 2.0f / a);
  return D;
}

__device__ __forceinline__ float G1_eval(int brdf, float c, float a, float* dc = nullptr, float* da = nullptr) {
  if (brdf == 0) {
    float a2 = a * a;
    float q = sqrtf(a2 + (1.0f - a2) * c * c);
    float s = c + q;
    if (dc) *dc = 2.0f * a2 / (q * s * s);
    if (da) *da = -2.0f * c / (s * s) * (a * (1.0f - c * c) / q);
    return 2.0f * c / s;
  }
  float s2 = 1.0f - c * c;
  if (!(s2 > 0.0f)) {
    if (dc) *dc = 0.0f;
    if (da) *da = 0.0f;
    return 1.0f;
  }
  float rs = sqrtf(s2);
  float x = c / (a * rs);
  float e = expf(-x * x);
  float G = 2.0f / (1.0f + erff(x) + e / (x * 1.7724538509055160f));
  float dGdx = G * G * e / (2.0f * 1.7724538509055160f * x * x);
  if (dc) *dc = dGdx / (a * s2 * rs);
  if (da) *da = dGdx * (-x / a);
  return G;
}

// Q = f(wi, wo) * cos(n, wi), RGB; zero unless both cosines are positive.
// (1 - wi.h)^5 of Schlick's Fresnel approximation F = ks + (1 - ks) x^5 (fr = 1); with fr = 0 the factor is
// held at ks, which x5 = 0 gives.
__device__ __forceinline__ float fresnel_x5(int fr, float cih) {
  if (!fr) return 0.0f;
  float x = 1.0f - cih, x2 = x * x;
  return x2 * x2 * x;
}

// f(wi, wo) cos(n, wi): kd/pi cos + F D G1(i) G1(o) / (4 cos_o), F per channel (held at ks, or Schlick with
// F0 = ks when fr = 1).
__device__ __forceinline__ float3 brdf_cos(int brdf, int fr, const Mat& m, float3 n, float3 wi, float3 wo) {
  float ci = dot3(n, wi), co = dot3(n, wo);
  if (!(ci > 0.0f) || !(co > 0.0f)) return mk3(0, 0, 0);
  float3 h = norm3(wi + wo);
  float ch = dot3(n, h);
  bool cl;
  float a = clamp_alpha(m.alpha, cl);
  float spec = D_eval(brdf, ch, a) * G1_eval(brdf, ci, a) * G1_eval(brdf, co, a) / (4.0f * co);
  float x5 = fresnel_x5(fr, dot3(wi, h));
  float kdc = ci * (1.0f / PI_F);
  return mk3(m.kd[0] * kdc + (m.ks[0] + (1.0f - m.ks[0]) * x5) * spec,
             m.kd[1] * kdc + (m.ks[1] + (1.0f - m.ks[1]) * x5) * spec,
             m.kd[2] * kdc + (m.ks[2] + (1.0f - m.ks[2]) * x5) * spec);
}

// One-sample lobe-mixture pdf (solid angle) of direction wi.
__device__ __forceinline__ float brdf_pdf(int brdf, const Mat& m, float3 n, float3 wi, float3 wo) {
  float ci = dot3(n, wi), co = dot3(n, wo);
  if (!(ci > 0.0f) || !(co > 0.0f)) return 0.0f;
  float3 h = norm3(wi + wo);
  float ch = dot3(n, h), woh = fabsf(dot3(wo, h));
  bool cl;
  float a = clamp_alpha(m.alpha, cl);
  float ps = lobe_prob(m);
  return (1.0f - ps) * ci * (1.0f / PI_F) + ps * D_eval(brdf, ch, a) * ch / (4.0f * woh);
}

// Orthonormal frame around n: t = (h x n)/|h x n|, b = n x t, helper axis h =
// (7, 9, 11)/16 (exact in binary, on no coordinate axis or plane), a second
// helper near n = +-h. Continuous in n elsewhere, so normals that lie exactly
// on a coordinate plane (symmetric meshes) get the same frame at any
// precision; the lobes are isotropic, so the frame changes no density.
__device__ __forceinline__ void onb(float3 n, float3& t, float3& b) {
  float3 c = cross3(mk3(0.4375f, 0.5625f, 0.6875f), n);
  float l2 = dot3(c, c);
  if (!(l2 > 1e-12f)) {
    c = cross3(mk3(0.6875f, -0.4375f, 0.5625f), n);
    l2 = dot3(c, c);
  }
  t = c * rsqrtf(l2);
  b = cross3(n, t);
}

// Returns the mixture pdf of the sampled direction wi; 0 = no valid sample.
__device__ __forceinline__ float brdf_sample(int brdf, const Mat& m, float3 n, float3 wo, float ul, float u1, float u2,
                                             float3& wi) {
  float3 t, b;
  onb(n, t, b);
  float ps = lobe_prob(m);
  if (ul < ps) {
    bool cl;
    float a = clamp_alpha(m.alpha, cl);
    float a2 = a * a;
    float tan2 = brdf == 0 ? a2 * u1 / (1.0f - u1) : -a2 * logf(1.0f - u1);
    float ch = rsqrtf(1.0f + tan2);
    float sh = sqrtf(fmaxf(0.0f, 1.0f - ch * ch));
    float sp, cp;
    sincosf(2.0f * PI_F * u2, &sp, &cp);
    float3 h = t * (sh * cp) + b * (sh * sp) + n * ch;
    wi = h * (2.0f * dot3(wo, h)) - wo;
  } else {
    // concentric square-to-disk map (Shirley and Chiu 1997), then project up
    float a = 2.0f * u1 - 1.0f, c = 2.0f * u2 - 1.0f;
    float x = 0.0f, y = 0.0f;
    if (a != 0.0f || c != 0.0f) {
      float r, ph;
      if (fabsf(a) > fabsf(c)) { r = a; ph = (PI_F * 0.25f) * (c / a); }
      else { r = c; ph = PI_F * 0.5f - (PI_F * 0.25f) * (a / c); }
      float sp, cp;
      sincosf(ph, &sp, &cp);
      x = r * cp; y = r * sp;
    }
    float z = sqrtf(fmaxf(0.0f, 1.0f - x * x - y * y));
    wi = t * x + b * y + n * z;
  }
  if (!(dot3(n, wi) > 0.0f)) return 0.0f;
  return brdf_pdf(brdf, m, n, wi, wo);
}

// Adjoint of Q = f(wi, wo) cos(n, wi) for an RGB output weight gw:
// accumulates dn, dwi (if non-null) and d params (kd_r, kd_g, kd_b, ks_r, ks_g, ks_b, alpha).
// With Schlick's factor (fr = 1), F_c = ks_c + (1 - ks_c) x^5, x = 1 - wi.h: dF_c/dks_c = 1 - x^5, and F
// moves with wi through wi.h: d(wi.h)/dwi = h + (wi - h (wi.h)) / |wi + wo| (wo is a fixed direction).
__device__ __forceinline__ void brdf_cos_adj(int brdf, int fr, const Mat& m, float3 n, float3 wi, float3 wo,
                                             float3 gw, float3& dn, float3* dwi, float dm[7]) {
  float ci = dot3(n, wi), co = dot3(n, wo);
  if (!(ci > 0.0f) || !(co > 0.0f)) return;
  float3 hu = wi + wo;
  float hl = len3(hu);
  float3 h = hu * (1.0f / hl);
  float ch = dot3(n, h);
  bool cl;
  float a = clamp_alpha(m.alpha, cl);
  float Dc, Da, Gic, Gia, Goc, Goa;
  float D = D_eval(brdf, ch, a, &Dc, &Da);
  float Gi = G1_eval(brdf, ci, a, &Gic, &Gia);
  float Go = G1_eval(brdf, co, a, &Goc, &Goa);
  float cih = dot3(wi, h);
  float x5 = fresnel_x5(fr, cih);
  float F0 = m.ks[0] + (1.0f - m.ks[0]) * x5, F1 = m.ks[1] + (1.0f - m.ks[1]) * x5,
        F2 = m.ks[2] + (1.0f - m.ks[2]) * x5;
  float gs = gw.x * F0 + gw.y * F1 + gw.z * F2;   // output weight times the lobe's colour
  float inv4co = 1.0f / (4.0f * co);
  float S = D * Gi * Go * inv4co;
  dm[0] += gw.x * ci * (1.0f / PI_F);
  dm[1] += gw.y * ci * (1.0f / PI_F);
  dm[2] += gw.z * ci * (1.0f / PI_F);
  dm[3] += gw.x * S * (1.0f - x5);
  dm[4] += gw.y * S * (1.0f - x5);
  dm[5] += gw.z * S * (1.0f - x5);
  if (!cl) dm[6] += gs * (Da * Gi * Go + D * Gia * Go + D * Gi * Goa) * inv4co;
  float dci = (gw.x * m.kd[0] + gw.y * m.kd[1] + gw.z * m.kd[2]) * (1.0f / PI_F) + gs * D * Gic * Go * inv4co;
  float dco = gs * D * Gi * (Goc * co - Go) * inv4co / co;
  float dch = gs * Dc * Gi * Go * inv4co;
  dn += wi * dci + wo * dco + h * dch;
  if (dwi) {
    float3 dh = n * dch;
    if (fr) {
      // dQ/d(wi.h) = -5 x^4 S sum_c gw_c (1 - ks_c); wi.h = wi . h reaches wi directly and through h
      float x = 1.0f - cih, x2 = x * x;
      float dcih = -5.0f * x2 * x2 * S *
                   (gw.x * (1.0f - m.ks[0]) + gw.y * (1.0f - m.ks[1]) + gw.z * (1.0f - m.ks[2]));
      *dwi += h * dcih;
      dh += wi * dcih;
    }
    float3 dhu = (dh - h * dot3(dh, h)) * (1.0f / hl);
    *dwi += n * dci + dhu;
  }
}

}  // namespace st

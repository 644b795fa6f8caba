// Stack-based traversal of the LBVH (closest hit and any hit).
//
// Internal node layout (64 bytes, four float4, read as 16-byte vector loads):
//   n0 = (lo_l.x, hi_l.x, lo_l.y, hi_l.y)
//   n1 = (lo_l.z, hi_l.z, lo_r.x, hi_r.x)
//   n2 = (lo_r.y, hi_r.y, lo_r.z, hi_r.z)
//   n3 = (child_l, child_r, -, -) as int bits; a child c < 0 is leaf ~c.
// Leaf i is the triangle record tri[3i..3i+2] = v0 (w = face id bits), v1, v2,
// stored in Morton order. Children that are leaves are intersected as soon as
// their box is hit; the far internal child is pushed. The first TRACE_SH
// entries of the stack live in shared memory (strided by block size), the
// rest in local memory.
#pragma once
#include "st_device.cuh"

namespace st {

constexpr int TRACE_SH = 16;
constexpr int TRACE_DEPTH = 64;
constexpr int ERR_STACK = 1;
constexpr int ERR_LOOP = 2;   // more node fetches than the tree has nodes: malformed hierarchy

struct TraceStats { int visits, tests; };

__device__ __forceinline__ float3 safe_inv(float3 d) {
  auto inv1 = [](float x) { return fabsf(x) > 1e-30f ? 1.0f / x : copysignf(1e30f, x); };
  return mk3(inv1(d.x), inv1(d.y), inv1(d.z));
}

// slab test of box [lo, hi]; returns entry distance or +inf on a miss
__device__ __forceinline__ float box_hit(float lx, float hx, float ly, float hy, float lz, float hz, float3 o,
                                         float3 inv, float tmax) {
  float tx0 = (lx - o.x) * inv.x, tx1 = (hx - o.x) * inv.x;
  float ty0 = (ly - o.y) * inv.y, ty1 = (hy - o.y) * inv.y;
  float tz0 = (lz - o.z) * inv.z, tz1 = (hz - o.z) * inv.z;
  float tn = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fmaxf(fminf(tz0, tz1), 0.0f));
  float tf = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fminf(fmaxf(tz0, tz1), tmax));
  // widen the far distance by 1 + 2*gamma(3) so rounding never culls a hit
  // (Ize, "Robust BVH Ray Traversal", JCGT 2013)
  return tn <= tf * 1.00000036f ? tn : __int_as_float(0x7f800000);
}

// ANY = stop at the first hit (shadow rays). Returns the face id or -1; t in tbest.
template <bool ANY, bool STATS>
__device__ __forceinline__ int trace_bvh(const float4* __restrict__ nodes, const float4* __restrict__ tri, int nf,
                                         float3 o, float3 d, float tmax, int exclude, float& tbest, int* sstack,
                                         int* err, TraceStats* ts) {
  RayPre rp = ray_pre(o, d);
  float3 inv = safe_inv(d);
  int best = -1;
  tbest = tmax;
  auto leaf = [&](int li) -> bool {
    float4 a = __ldg(&tri[3 * li]);
    int fid = __float_as_int(a.w);
    if (STATS) ts->tests++;
    if (fid == exclude) return false;
    float4 b = __ldg(&tri[3 * li + 1]);
    float4 c = __ldg(&tri[3 * li + 2]);
    float t = tri_test(rp, xyz(a), xyz(b), xyz(c), ANY ? tmax : tbest * 1.0000001f + 1e-30f);
    if (t > 0.0f) {
      if (ANY) { best = fid; tbest = t; return true; }
      if (t < tbest || (t == tbest && fid < best)) { tbest = t; best = fid; }
    }
    return false;
  };
  if (nf == 1) {
    leaf(0);
    return best;
  }
  int local[TRACE_DEPTH - TRACE_SH];
  const int bd = blockDim.x;
  int sp = 0;
  int node = 0;
  int budget = nf;  // a well-formed tree fetches each of its nf - 1 internal nodes at most once
  for (;;) {
    if (--budget < 0) { atomicOr(err, ERR_LOOP); return best; }
    const float4* np = nodes + 4 * node;
    float4 n0 = __ldg(np), n1 = __ldg(np + 1), n2 = __ldg(np + 2), n3 = __ldg(np + 3);
    if (STATS) ts->visits++;
    float tl = box_hit(n0.x, n0.y, n0.z, n0.w, n1.x, n1.y, o, inv, tbest);
    float tr = box_hit(n1.z, n1.w, n2.x, n2.y, n2.z, n2.w, o, inv, tbest);
    int cl = __float_as_int(n3.x), cr = __float_as_int(n3.y);
    bool hl = tl != __int_as_float(0x7f800000), hr = tr != __int_as_float(0x7f800000);
    if (hl && cl < 0) { if (leaf(~cl) && ANY) return best; hl = false; }
    if (hr && cr < 0) { if (leaf(~cr) && ANY) return best; hr = false; }
    if (hl && hr) {
      int nearc = tl <= tr ? cl : cr, farc = tl <= tr ? cr : cl;
      if (sp >= TRACE_DEPTH) { atomicOr(err, ERR_STACK); return best; }
      if (sp < TRACE_SH) sstack[sp * bd] = farc; else local[sp - TRACE_SH] = farc;
      ++sp;
      node = nearc;
    } else if (hl) {
      node = cl;
    } else if (hr) {
      node = cr;
    } else {
      if (sp == 0) break;
      --sp;
      node = sp < TRACE_SH ? sstack[sp * bd] : local[sp - TRACE_SH];
    }
  }
  return best;
}

}  // namespace st
